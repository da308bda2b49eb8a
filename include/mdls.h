/*
 * mdls.h -- C ABI of the B300 (sm_103a) library for the MDFIS local-search hot path of
 * Lei & Hao, "A GPU-Accelerated Hybrid Method for a Class of Multi-Depot Vehicle Routing
 * Problems" (MDFIHA-ETGA).
 *
 * The library evaluates whole neighbourhoods of Relocate, Swap, 2-opt*, Depot-Insert and
 * Depot-Replace (Section 3.2.2) for many solutions at once, scores every move under the
 * multi-penalty evaluation function F (Eq. 2, detailed in Eq. A1) from per-route prefix and
 * suffix segment summaries, selects a leader and non-conflicting followers (Section 3.2.5),
 * applies them and rebuilds only the touched routes (Alg. 2, "update tensor T_s").
 *
 * Conventions shared by every call:
 *   - Every call returns md_status.  On failure md_last_error() returns a message describing
 *     the first error of the calling thread (thread-local; valid until the next failing call).
 *   - Handles are opaque.  The library copies every host input it needs and owns all the
 *     device memory behind a handle until the matching *_destroy call.
 *   - Device work is stream ordered on `stream`, a cudaStream_t passed as void* (NULL = the
 *     legacy default stream).  Calls that return host data synchronise that stream.
 *   - Node ids: depots are 0..n_depots-1, customers n_depots..n_depots+n_customers-1; at most
 *     16384 nodes (move ids pack two node ids in 14 bits each).
 *   - Fixed point: every distance and time is an integer equal to round(scale * value), with
 *     distances rounded half away from zero from the FP64 Euclidean distance; travel time
 *     equals distance (t_ij = c_ij).  Demands and capacities are plain integers.
 *   - Move ids: op << 32 | u << 18 | v << 4 | variant (see MD_OP_*); they are independent of
 *     how routes are laid out in memory and break every tie.
 */
#ifndef MDLS_H
#define MDLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum md_status {
    MD_OK = 0,
    MD_ERR_ARG = 1,      /* invalid argument or input data */
    MD_ERR_CUDA = 2,     /* a CUDA runtime call failed */
    MD_ERR_CAPACITY = 3, /* a route or buffer capacity was exceeded */
    MD_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
    MD_ERR_STATE = 5,    /* calls made in an order the object does not allow */
    MD_ERR_BOUNDS = 6    /* a build with MD_DEBUG_BOUNDS found a device-side index out of range */
} md_status;

/* Instance variant flags (Section 1: MDVRP, MDVRPTW, MDOVRP). */
#define MD_VARIANT_TW 1u        /* time windows: time-warp penalty V1 */
#define MD_VARIANT_OPEN 2u      /* open routes: no return arc, no closure term */
#define MD_VARIANT_SYMMETRIC 4u /* 2-node sequences may be reversed (Section 3.2.2) */

/* Operators (Section 3.2.2).  Variants per operator:
 *   RELOCATE  0: seq(u) of 1 node after v        1: 1 node before v (v first on its route)
 *             2: seq(u) of 2 nodes after v       3: 2 nodes before v (v first)
 *             4: 2 nodes reversed after v        5: 2 nodes reversed before v (v first)
 *             (4 and 5 only on symmetric instances)
 *   SWAP      (|seq(u)|, |seq(v)|) = 0:(1,1) 1:(2,1) 2:(1,2) 3:(2,2); on symmetric instances
 *             also 4:(2r,1) 5:(1,2r) 6:(2r,2) 7:(2,2r) 8:(2r,2r), r = reversed where placed
 *   TWO_OPT_STAR  0: head(..u) + tail(v..) and head(..pred v) + tail(succ u..)
 *   DEPOT_INSERT  u = c_k, v = depot d: [ds..c_k, d] and [d, c_k+1..de], 1 <= k < L
 *   DEPOT_REPLACE u = first customer of the route, v = depot d, variant = case 0: departure,
 *                 1: arrival, 2: both; one move per (route, d): the best case by (dF, case)
 */
#define MD_OP_RELOCATE 0
#define MD_OP_SWAP 1
#define MD_OP_TWO_OPT_STAR 2
#define MD_OP_DEPOT_INSERT 3
#define MD_OP_DEPOT_REPLACE 4
#define MD_OP_TWO_OPT 5  /* intra-route 2-opt (Section 3.2.2): on the route holding u and v, the
                            customers from the one after the earlier of them through the later
                            are reversed (at least two); symmetric instances without time windows
                            only -- no moves otherwise, as the paper leaves 2-opt out with time
                            windows.  Variant 0. */
#define MD_N_OPS 6

/* md_eval_neighborhood flags */
#define MD_EVAL_DUMP 1u      /* also write every scored move to the moves object's dump list */
#define MD_EVAL_FOLLOWERS 2u /* record the best follower of every route pair (multi-move) */

/* md_apply_and_rebuild flags */
#define MD_APPLY_UPDATE_LAMBDA 1u /* adapt lambda after an accepted step (Section 3.2.1) */

typedef struct md_instance md_instance;
typedef struct md_solutions md_solutions;
typedef struct md_moves md_moves;

/* Problem data of Section 1 (Eq. 1).  All arrays have n_depots + n_customers entries, depots
 * first; the library copies them.  Times (service, tw_early, tw_late, D) are fixed point
 * (already multiplied by `scale`); coordinates are plain doubles and are scaled when the
 * distances are built.  Depot entries of demand and service are ignored (taken as 0).
 * tw_early / tw_late may be NULL when MD_VARIANT_TW is not set. */
typedef struct md_instance_desc {
    int32_t n_depots;
    int32_t n_customers;
    const double *x;
    const double *y;
    const int32_t *demand;
    const int32_t *service;
    const int32_t *tw_early;
    const int32_t *tw_late;
    int32_t Q;       /* vehicle capacity */
    int32_t N_V;     /* vehicles per depot */
    int32_t D;       /* maximum route duration, fixed point; 0 = no limit */
    uint32_t variant;/* MD_VARIANT_* */
    double scale;    /* fixed-point factor, e.g. 100 */
    int32_t theta;   /* granular neighbours per customer (Section 3.2.3); 0 = all customers */
} md_instance_desc;

/* One scored move, as written by MD_EVAL_DUMP.  Deltas are new minus old for: total distance D,
 * time warp (V1 before Gamma), load excess (V2 before Theta/Q), duration excess (V3 before
 * Theta/D), depot violations (V4 before Theta: closures plus vehicle excess).  dF combines
 * them in FP64 as (((dD + w1 dTW) + w2 dLoad) + w3 dDur) + w4 dV4 with w1 = lambda1 Gamma,
 * w2 = lambda2 Theta / Q, w3 = lambda3 Theta / D (0 without D), w4 = lambda4 Theta (Eq. A1). */
typedef struct md_move {
    uint64_t id;
    int64_t dD, dTW, dLoad, dDur, dV4;
    double dF;
    int32_t sol;   /* solution index */
    int32_t pad;
} md_move;

/* Settings of the MDFIS descent (Alg. 2). */
typedef struct md_config {
    int32_t n_ops;          /* operators per pass, 1..8 */
    int32_t max_pass;       /* search depth delta: passes of the while loop of Alg. 2 */
    const uint8_t *op_perm; /* host [n_sol * max_pass * n_ops]: the operator order of every pass
                               (Alg. 2 draws a random permutation; the caller supplies the draws) */
    const float *lambda0;   /* host [n_sol * 4] initial lambda, or NULL for (1, 1, 1, 1) */
    int32_t multi_move;     /* 1: leader + followers (Section 3.2.5); 0: leader only */
    int32_t lambda_update;  /* 1: adapt lambda after every accepted step (kappa = 0.5) */
    int32_t use_graph;      /* 1: replay one captured CUDA graph per pass */
    int32_t poll_every;     /* passes between host checks of the per-solution done flags */
    int32_t op_perm_device; /* 1: op_perm points to device memory (no host copy per call) */
    int32_t time_eval;      /* 1: time every evaluation launch with CUDA events (md_stats.eval_ms) */
    int32_t n_groups;       /* > 1: solutions advance in this many groups on concurrent streams
                               (needs a non-NULL stream); results do not depend on it */
    int32_t sweep_every;    /* > 0: every sweep_every-th step of a solution evaluates the full
                               neighbourhood (all customers) instead of the neighbour lists; the
                               fallback of pruned lists.  A pass that applies nothing is then
                               followed by a verification pass whose steps evaluate the full
                               neighbourhood until one applies a move; the descent ends only
                               when a verification pass applies nothing (or at max_pass).
                               0: never (the descent ends at the first pass applying nothing) */
    int32_t persistent;     /* 1: the whole descent in ONE persistent launch: each solution's
                               evaluation tiles and steps go through device-side task queues as
                               soon as they can run (the last tile of an evaluation queues its
                               step, a step queues the next evaluation's tiles), so every
                               solution advances on its own and steps overlap other solutions'
                               evaluation; use_graph, poll_every and n_groups are then unused,
                               and time_eval times the launch.  Needs a non-NULL stream.  Same
                               results as 0.  MD_ERR_TIMEOUT if a bounded wait gives up. */
    int32_t wide_step;      /* graph form (persistent = 0; in md_batch_descend the instances that
                               run solo) only: how a step selects, applies and
                               rebuilds.  1: spread over the grid in four launches (one CTA per
                               solution selects, one warp per selected move applies it, one warp
                               per touched route rebuilds it, one CTA per solution finishes);
                               -1: one CTA per solution does it all; 0: 1 when the solutions
                               have at least 256 route slots, else -1.  Same results. */
    int32_t wait_limit;     /* persistent descent: polls without progress before one of its
                               device-side waits gives up (the kernel then stops every CTA and
                               the call returns MD_ERR_TIMEOUT); 0: the default, 2^22 (about a
                               second).  Failure detection is tested with a budget of 1. */
} md_config;

/* Totals over all solutions of one md_descend call. */
typedef struct md_stats {
    int64_t moves_scored;   /* scored move tuples (op, u, v, variant) */
    int64_t steps;          /* operator evaluations (solution x operator) */
    int64_t accepted_steps; /* steps that applied a leader */
    int64_t applied_moves;  /* leaders + followers applied */
    int64_t passes_max;     /* largest number of passes any solution ran */
    int64_t launches;       /* kernels launched by the call */
    int64_t eval_launches;  /* evaluation kernel launches */
    double eval_ms;         /* summed device time of the evaluation launches (time_eval = 1) */
    int64_t moves_by_op[MD_N_OPS]; /* scored move tuples per operator */
    int64_t moves_exact;    /* moves whose concatenations were formed: on full neighbourhoods the
                               others are decided by an exact lower bound (neither leader nor
                               follower), so moves_scored - moves_exact were counted unformed */
    int64_t moves_exact_by_op[MD_N_OPS];
} md_stats;

/* Message for the calling thread's last failing call ("" if none). */
const char *md_last_error(void);

/* Builds the instance on the device (Section 1; Eq. A1 for Theta = 2 max c - min c and
 * Gamma = sum c / sum t; Section 3.2.3 for the neighbour lists: edge (u,v) is pruned when
 * e_u + s_u + t_uv > l_v (time windows only), then the theta candidates with the smallest
 * eta_uv of Eq. 3 (alpha = 1, beta = 10; ties by node id) are kept).
 * MD_ERR_ARG: null pointers, sizes out of range (n_depots < 1, n_customers < 1, more than
 * 16384 nodes, Q < 1, N_V < 1, theta < 0), windows with tw_early > tw_late or above 2^30. */
md_status md_instance_create(const md_instance_desc *desc, md_instance **out);
md_status md_instance_destroy(md_instance *inst);

/* Theta (int64) and Gamma (FP64) of Eq. A1. */
md_status md_instance_params(const md_instance *inst, int64_t *theta_big, double *gamma);

/* Copies the distance matrix (int32, [n_nodes * n_nodes], row-major) to host memory. */
md_status md_instance_read_dist(const md_instance *inst, int32_t *host_out);

/* Copies the neighbour lists: host_nbr [n_customers * theta] node ids (row = customer index),
 * host_cnt [n_customers] list lengths.  MD_ERR_STATE when theta = 0. */
md_status md_instance_read_neighbors(const md_instance *inst, int32_t *host_nbr, int32_t *host_cnt);

/* Recomputes the granular neighbour lists with a new width theta (ranking of
 * md_instance_create, Section 3.2.3 / Eq. 3); theta = 0 switches to the full neighbourhood.  Takes
 * effect for evaluations launched afterwards. */
md_status md_instance_build_neighbors(md_instance *inst, int32_t theta);

/* Installs caller-chosen neighbour lists: nbr [n_customers * theta] node ids (row = customer
 * index), cnt [n_customers] list lengths (<= theta).  Every entry must be a customer other than
 * the row's own (MD_ERR_ARG otherwise).  Used for learned candidate lists. */
md_status md_instance_set_neighbors(md_instance *inst, const int32_t *nbr, const int32_t *cnt, int32_t theta);

/* Allocates n_sol solutions of the instance, each with r_slots route slots of up to k_max
 * customers.  A route slot holds one route [ds, c_1..c_L, de] (Eq. 1 notation) with its
 * per-customer prefix/suffix segment summaries (Section 3.2.2, sequence concatenation).
 * MD_ERR_ARG when k_max is so large that int32 summaries could overflow. */
md_status md_solutions_create(const md_instance *inst, int32_t n_sol, int32_t r_slots,
                              int32_t k_max, md_solutions **out);
md_status md_solutions_destroy(md_solutions *sols);

/* Loads routes from host memory: route i of the flattened list is
 * route_nodes[route_offsets[i] .. route_offsets[i+1]) = [ds, c_1..c_L, de] (de is kept but has
 * no meaning for open routes); solution s owns the next routes_per_sol[s] routes.  Validates
 * that every customer appears exactly once per solution and that every route is non-empty with
 * depots at both ends (MD_ERR_ARG), and that it fits the slots (MD_ERR_CAPACITY).  Resets the
 * per-solution lambda to (1, 1, 1, 1) and rebuilds every summary on the device. */
md_status md_solutions_load(md_solutions *sols, const int32_t *route_nodes,
                            const int64_t *route_offsets, const int32_t *routes_per_sol,
                            void *stream);

/* Device-to-device copy of the routes of src into dst (same instance and shape), followed by a
 * rebuild of every summary; lambda reset to (1, 1, 1, 1). */
md_status md_solutions_copy(md_solutions *dst, const md_solutions *src, void *stream);

/* Exports the routes in the md_solutions_load layout (slot order).  MD_ERR_CAPACITY when
 * node_cap or route_cap is too small. */
md_status md_solutions_read(md_solutions *sols, int32_t *route_nodes, int64_t *route_offsets,
                            int32_t *routes_per_sol, int64_t node_cap, int64_t route_cap,
                            void *stream);

/* Per solution: comps [n_sol * 8] = D, TW, LoadEx, DurEx, closures, vehicle excess, V4, routes
 * (int64, Eq. A1 before the weights) and F [n_sol] under the solution's current lambda. */
md_status md_solution_cost(md_solutions *sols, int64_t *comps, double *F, void *stream);

/* Current lambda [n_sol * 4] (FP32). */
md_status md_solutions_lambda(md_solutions *sols, float *lambda, void *stream);

/* Per-customer summaries, for tests: pre/suf [n_sol * n_customers * 8] int32 with
 * pre = {dist, load, dur, tw, E, L, route slot, position} of [ds..c] and
 * suf = {dist, load, dur, tw, E, L, pred node, succ node} of [c..de] (open routes: [c..c_L]). */
md_status md_solutions_read_summaries(md_solutions *sols, int32_t *pre, int32_t *suf, void *stream);

/* Scratch for one evaluation: per-block leader candidates, the follower table (one entry per
 * route pair), the selection and an optional dump list of dump_capacity moves. */
md_status md_moves_create(const md_solutions *sols, int64_t dump_capacity, md_moves **out);
md_status md_moves_destroy(md_moves *moves);

/* Evaluates the whole neighbourhood of operator ops[s] for every solution s (ops[s] < 0 skips
 * it): every valid move (u, v, variant) of Section 3.2.2 over u's neighbour list (or all
 * customers when theta = 0), plus every route x depot of the depot operators, each scored from
 * the segment summaries (Eq. A1) with dF as in md_move.  Records per solution the leader (the
 * smallest dF < 0, ties by id) and, with MD_EVAL_FOLLOWERS, the best follower (dD < 0 and no
 * change in any penalty term, Section 3.2.5) of every route pair.  lambda: host [n_sol * 4] to
 * set before evaluating, or NULL to keep the current values.
 * MD_ERR_CAPACITY when MD_EVAL_DUMP overflows the dump list (the list then holds a prefix). */
md_status md_eval_neighborhood(md_solutions *sols, const int32_t *ops, const float *lambda,
                               uint32_t flags, md_moves *moves, void *stream);

/* Results of the last evaluation: leader id (0 when none) and dF per solution, and the number
 * of scored move tuples per solution. */
md_status md_moves_read_leaders(md_moves *moves, uint64_t *ids, double *dF, int64_t *n_scored,
                                void *stream);

/* The dump list of the last MD_EVAL_DUMP evaluation, in no particular order. */
md_status md_moves_read_dump(md_moves *moves, md_move *host_out, int64_t cap, int64_t *n_out,
                             void *stream);

/* Leader-follower selection (Section 3.2.5): per solution the leader, then the followers in
 * ascending (dD, id) order, each taken when none of its routes is already claimed.  Computed
 * on the device by rounds of per-route minimum claims, which yields the same set as that
 * sequential greedy.  multi_move = 0 keeps the leader only. */
md_status md_select_multimove(md_solutions *sols, md_moves *moves, int32_t multi_move,
                              void *stream);

/* The selection: ids [n_sol * cap] (leader first), counts [n_sol]. */
md_status md_selection_read(md_moves *moves, uint64_t *ids, int32_t *counts, int32_t cap,
                            void *stream);

/* Applies the selected moves (route-disjoint) and rebuilds the summaries of the touched routes
 * only; an emptied route is deleted and Depot-Insert takes a free slot.  With
 * MD_APPLY_UPDATE_LAMBDA, lambda_i is divided by kappa = 0.5 where term i is violated after
 * the step and multiplied by it otherwise, kept in [2^-16, 2^16] (Section 3.2.1); lambda_out
 * (host [n_sol * 4], may be NULL) receives the values.  MD_ERR_CAPACITY when a new route does
 * not fit k_max or no free slot is left (that move is skipped). */
md_status md_apply_and_rebuild(md_solutions *sols, md_moves *moves, uint32_t flags,
                               float *lambda_out, void *stream);

/* MDFIS descent (Alg. 2) of every solution: per pass, the operators in the order of op_perm;
 * each step evaluates, selects and applies on the device; a solution stops after a pass that
 * applied nothing or after max_pass passes.  The host only polls the done flags. */
md_status md_descend(md_solutions *sols, const md_config *cfg, md_stats *out, void *stream);

/* Per-solution counters of the last md_descend: [n_sol * 5] = moves scored, steps, accepted
 * steps, applied moves, passes. */
md_status md_solutions_stats(md_solutions *sols, int64_t *per_sol, void *stream);

/* Repair insertion rules (Section 3.3, the insertion step of the route-exchange crossover).
 * The cost of inserting customer u after position k of a route is the change of its travel
 * distance, c(c_k, u) + c(u, c_{k+1}) - c(c_k, c_{k+1}) (one arc c(c_L, u) after the last
 * customer of an open route); an insertion is feasible when the new route has no load excess,
 * no time warp and no duration excess.
 *   MD_INSERT_FBI  feasible best insertion: the cheapest feasible insertion of any unrouted
 *                  customer, ties by the customer's place in the list, then route slot, then
 *                  position;
 *   MD_INSERT_IBI  infeasible best insertion: the same over every insertion;
 *   MD_INSERT_FRI  feasible regret insertion: per customer, its best feasible insertion and its
 *                  best feasible insertion into any other route; the customer of largest regret
 *                  (their cost difference, unbounded when no other route takes it) goes first,
 *                  ties by the cheaper best insertion, then the list; it goes to its best
 *                  insertion;
 *   MD_INSERT_IRI  infeasible regret insertion: the same over every insertion.
 * FBI and FRI open a route [d, u, d] for the first listed customer when no listed customer has
 * a feasible insertion: d is the depot nearest to u (c(d, u) + c(u, d); c(d, u) for open
 * routes) among those with fewer than N_V routes, else among all, ties by index.  IBI and IRI
 * open a route only when the solution has none.  New routes take the first free slot. */
#define MD_INSERT_FBI 0
#define MD_INSERT_IBI 1
#define MD_INSERT_FRI 2
#define MD_INSERT_IRI 3

/* Loads partial solutions and inserts the unrouted customers of solution s by rules[s]
 * (MD_INSERT_*; host int32 [n_sol]), one thread-block cluster per solution on the device (its
 * CTAs split the solution's list and pick each insertion together; the cluster size follows
 * md_solutions_set_repair_split); on return sols holds complete solutions with every summary
 * and total rebuilt (lambda reset to 1), ready for md_descend.
 *   route_nodes / route_offsets / routes_per_sol: host, the md_solutions_load layout, except
 *     that a solution may have no route (routes_per_sol[s] = 0) and leaves customers out;
 *     route_nodes and route_offsets may be NULL when no solution has a route;
 *   unrouted: host int32, solution s's unrouted customers at unrouted[unrouted_offsets[s] ..
 *     unrouted_offsets[s + 1]) in order of preference (the tie-break); unrouted_offsets: host
 *     int64 [n_sol + 1], unrouted_offsets[0] = 0;
 *   order: optional host int32 [unrouted_offsets[n_sol]], receives per solution the customers in
 *     the order they were inserted.
 * MD_ERR_ARG unless every customer appears exactly once per solution (in a route or in its
 * list) and the routes are well formed; MD_ERR_CAPACITY when a route would exceed k_max or a
 * new route finds no free slot (the solution then holds a partial repair).  Synchronises the
 * stream. */
md_status md_repair_insert(md_solutions *sols, const int32_t *rules, const int32_t *route_nodes,
                           const int64_t *route_offsets, const int32_t *routes_per_sol,
                           const int32_t *unrouted, const int64_t *unrouted_offsets, int32_t *order,
                           void *stream);

/* How md_repair_insert spreads a solution over CTAs: one CTA per per_cta listed customers of the
 * longest list, at most 16 (0: 128, the default).  A cluster size the device cannot place is not
 * used; among the rest the call picks the one that finishes every solution in the fewest waves
 * per CTA.  Results do not depend on it.  MD_ERR_ARG on a null set or per_cta < 0. */
md_status md_solutions_set_repair_split(md_solutions *sols, int32_t per_cta);

/* The route exchange of DCREX (Alg. 3, Section 3.3) for one offspring, on the host (no device
 * work): from the main member's routes and, in the given order, the routes of other members of
 * a population, builds the offspring's partial solution and lists its unrouted customers.
 * Route pairs (R_i, R_j) -- R_i a route of the main member still in the offspring, R_j a route
 * of the current other member -- score N^R + N^M + 10 N^C - E^I, where E^I counts R_j's distinct
 * edges the offspring does not have, N^R R_i's customers R_j does not visit, N^M R_j's customers
 * the offspring visits outside R_i, and N^C R_j's customers visited by routes introduced earlier
 * in this call.  One of the five lowest scores (ties by i, then j) is drawn uniformly, R_j
 * replaces R_i, and E^I + N^R + N^M is summed; the exchange goes on while the sum is below
 * smin = degree/20 (n_customers + m) or at least smax = (degree+1)/20 (n_customers + m) (m: the
 * main member's routes) and stops in between, or when no route of the main member is left or a
 * member has no route.  Redundant customers then stay in the earliest-introduced route that
 * visits them; routes left empty are dropped.  Edges are undirected pairs of consecutive nodes,
 * depots included; open routes (open_routes != 0) have no return edge, and a closed route
 * [d, c, d] has one edge.
 *   nodes / offsets / routes_per_member: host, every member's routes in the md_solutions_load
 *     layout (routes of member k follow those of member k - 1; each route starts and ends at a
 *     depot and visits at least one customer; a member visits a customer at most once);
 *   main_member: the main parent's index; others: host int32 [n_others], member indices in the
 *     order they are visited;
 *   degree: the diversity degree, 0..19;
 *   stream: host uint64 [2], {state, counter} of a counter-based SplitMix64 stream: a draw is
 *     the high 32 bits x of mix(state + counter' * 0x9E3779B97F4A7C15) with counter' = counter
 *     + 1, mapped to (x * span) >> 32; the call advances counter by its draws (one per
 *     exchanged route);
 *   out_nodes: host int32, room for n_customers + 2 m nodes; out_offsets: host int64 [m + 1];
 *     out_routes receives the offspring's routes (in the main member's route order, an
 *     exchanged route in the place of the one it replaced);
 *   unrouted: host int32 [n_customers], the customers in no route, increasing; n_unrouted their
 *     count.
 * MD_ERR_ARG on a null pointer, an index or degree out of range, or malformed routes. */
md_status md_dcrex(const int32_t *nodes, const int64_t *offsets, const int32_t *routes_per_member,
                   int32_t n_members, int32_t main_member, const int32_t *others, int32_t n_others,
                   int32_t degree, int32_t n_depots, int32_t n_customers, int32_t open_routes,
                   uint64_t *stream, int32_t *out_nodes, int64_t *out_offsets, int32_t *out_routes,
                   int32_t *unrouted, int32_t *n_unrouted);

/* Batches of instances of uneven size.  A batch groups solution sets of different instances
 * (each from md_solutions_create/load on the same device, each still owned by the caller) so
 * that every solution of every instance advances with ONE evaluation launch and ONE select/apply
 * launch per descent step (Alg. 2), replayed from a CUDA graph per pass: the evaluation launch is
 * persistent, its blocks walking a work list of (instance, solution, tile) with the largest
 * instances first.  MD_ERR_ARG on null or empty input. */
typedef struct md_batch md_batch;
md_status md_batch_create(md_solutions *const *sols, int32_t n, md_batch **out);
md_status md_batch_destroy(md_batch *batch);

/* Autotuner of the batch's tile shapes: per instance, the customer parts per warp of an
 * evaluation tile (1, 2 or 4) and, for an instance without neighbour lists, the warps that share
 * one customer's candidates (1, 2, 4 or 8, at most n_customers / 256), timed with CUDA events on
 * that instance alone, and whether the instance runs solo (md_batch_solo); then the persistent
 * grid (1, 2, 4 or 8 blocks per SM), timed on the instances left in the batched launch.  Uses the loaded solutions and sets every solution's operator to a fixed mix for the
 * timings.  Results only change speed. */
md_status md_batch_tune(md_batch *batch, void *stream);

/* The chosen shapes (caller order, [n] each; any pointer may be NULL): upw customer parts per
 * warp, wpc warps per customer, grid blocks of the evaluation launch. */
md_status md_batch_tuning(const md_batch *batch, int32_t *upw, int32_t *wpc, int32_t *grid);

/* Sets the shapes by hand (host arrays [n] in caller order; NULL keeps the current ones; grid
 * <= 0 keeps it): upw >= 1; wpc in 1..8, above 1 only for an instance without neighbour lists
 * and at most n_customers / 256.  MD_ERR_ARG otherwise (nothing changed).  Results only change
 * speed. */
md_status md_batch_set_tuning(md_batch *batch, const int32_t *upw, const int32_t *wpc, int32_t grid);

/* Which instances run on their own (caller order, host array [n]; 1 = solo): a solo instance
 * keeps its single-instance evaluation and select/apply launches (as md_descend would make them)
 * on a stream of its own, forked from the batch's stream inside the same graph, instead of
 * joining the batched launches.  md_batch_tune sets an instance solo when its own evaluation
 * launch is faster than the batched one on it alone; none is solo before.  md_batch_set_solo
 * sets the flags by hand (nonzero = solo).  MD_ERR_ARG on a null argument.  Results only change
 * speed. */
md_status md_batch_solo(const md_batch *batch, int32_t *solo);
md_status md_batch_set_solo(md_batch *batch, const int32_t *solo);

/* MDFIS descent (Alg. 2) of every solution of every instance, as md_descend per instance would
 * do it (identical results).  cfg->op_perm covers the solutions of all instances in the order
 * they were given to md_batch_create ([sum n_sol * max_pass * n_ops]); cfg->lambda0 likewise
 * ([sum n_sol * 4]) or NULL.  cfg->n_groups is ignored. */
md_status md_batch_descend(md_batch *batch, const md_config *cfg, md_stats *out, void *stream);

/* Learned move-proposal pruner (not in the paper: an extension that replaces the static
 * granular lists of Section 3.2.3 by learned ones; every kept candidate is still evaluated exactly,
 * and md_config.sweep_every supplies the periodic full sweep that catches what the lists miss).
 * Model: 32 pair features -> 128 -> ReLU -> 128 -> ReLU -> 1 logit.  Parameters, FP32, in this
 * order: W1 [128 x 32] (row = hidden unit), b1 [128], W2 [128 x 128], b2 [128], w3 [128], b3 [1]
 * (MD_PRUNER_PARAMS values).  Inference runs on the tensor cores with BF16 operands and FP32
 * accumulation; training keeps FP32 master weights with Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * The features of a pair (u, v) depend on the instance only. */
#define MD_PRUNER_PARAMS 20865
typedef struct md_pruner md_pruner;
md_status md_pruner_create(const float *params, md_pruner **out);
md_status md_pruner_destroy(md_pruner *pruner);
md_status md_pruner_params(md_pruner *pruner, float *params);

/* The 32 features of every (customer, listed candidate) pair of the instance's current lists:
 * feats [n_customers * theta * 32] (zeros for empty list slots). */
md_status md_pruner_features(md_pruner *pruner, md_instance *inst, float *feats, void *stream);

/* Logits of every (customer, listed candidate) pair: scores [n_customers * theta] (-inf for empty
 * slots). */
md_status md_pruner_score(md_pruner *pruner, md_instance *inst, float *scores, void *stream);

/* Scores the instance's current lists (the candidate pool, e.g. from md_instance_build_neighbors)
 * and installs, per customer, the k best candidates by (score descending, node id ascending) as
 * the instance's neighbour lists (theta becomes k). */
md_status md_pruner_prune(md_pruner *pruner, md_instance *inst, int32_t k, void *stream);

/* Trains on every (customer, listed candidate) pair of the instance's current lists, with labels
 * [n_customers * theta] (1: the pair took part in a selected move of a plain descent): `epochs`
 * passes in order, in mini-batches of `batch` pairs (a multiple of 32), binary cross-entropy
 * with positive pairs weighted by pos_weight, Adam with learning rate lr.  mean_loss (may be
 * NULL) receives the weighted mean loss of the last epoch. */
md_status md_pruner_train(md_pruner *pruner, md_instance *inst, const uint8_t *labels, int32_t epochs,
                          int32_t batch, float lr, float pos_weight, float *mean_loss, void *stream);

/* ---------------------------------------------------------------------------------------------
 * One solution split over ranks by customer (multi-GPU: the evaluation of a large solution shared
 * by several GPUs, one exchange per descent step).  The leader-follower update (Section 3.2.5)
 * needs from an evaluation only its leader (the smallest dF < 0) and, for every route pair, the
 * best follower: each rank evaluates the customers of its range (md_eval_range), exports that
 * summary (md_moves_export), the ranks all-gather it, every replica merges it (the smallest leader
 * by (dF, id); per route pair the smallest follower key; the summed scored counts) and imports it
 * (md_moves_import), then md_select_multimove and md_apply_and_rebuild run the identical selection
 * and apply on every replica, which therefore stay identical.
 * ------------------------------------------------------------------------------------------- */

/* A solution's best move of one evaluation. */
typedef struct md_leader {
    uint64_t id;      /* op << 32 | u << 18 | v << 4 | variant; 0 when valid = 0 */
    double dF;        /* its penalised delta (FP64) */
    uint32_t routes;  /* its route slots rA | rB << 16 */
    int32_t valid;    /* 1: a move with dF < 0 exists */
    int64_t scored;   /* moves scored by the evaluation for this solution */
} md_leader;

/* md_eval_neighborhood restricted to the customers u of indices c0 .. c1 - 1 (customer index =
 * node id - n_depots): only moves keyed by those u are scored.  Every other argument as
 * md_eval_neighborhood.  MD_ERR_ARG unless 0 <= c0 <= c1 <= n_customers. */
md_status md_eval_range(md_solutions *sols, const int32_t *ops, int32_t c0, int32_t c1, const float *lambda,
                        uint32_t flags, md_moves *moves, void *stream);

/* The last evaluation's leader of solution sol and its follower-table entries: pairs[k] =
 * i * r_slots + j (i <= j route slots), keys[k] = (dD ^ 0x80000000) << 32 | 32-bit move id of the
 * pair's best follower, k < n_out; cap: the arrays' length.  Empties the solution's table.  Host
 * buffers.  MD_ERR_CAPACITY (after writing cap entries) when n_out > cap; MD_ERR_STATE before an
 * evaluation. */
md_status md_moves_export(md_moves *moves, int32_t sol, md_leader *leader, uint32_t *pairs, uint64_t *keys,
                          int64_t cap, int64_t *n_out, void *stream);

/* Installs a merged summary for solution sol (the format of md_moves_export): the leader, n
 * follower entries with distinct pairs, and leader->scored as the scored count; the solution's
 * operator is the one of its last evaluation.  md_select_multimove may follow.  Host buffers.
 * MD_ERR_ARG for a pair outside the table, MD_ERR_CAPACITY for more entries than the table
 * lists. */
md_status md_moves_import(md_moves *moves, int32_t sol, const md_leader *leader, const uint32_t *pairs,
                          const uint64_t *keys, int64_t n, void *stream);

/* Failure detection of the tensor-core scoring (md_pruner_score / md_pruner_prune): the number of
 * polls a wait for the tensor cores makes before it gives up (0: every wait gives up at once);
 * a negative value restores the default (2^20).  A wait that gives up sets the pruner's error
 * flag, lets the MMAs in flight finish (a wait of the default length) before the CTA releases its
 * tensor memory, and stops the CTA; the call then returns MD_ERR_TIMEOUT.  Not part of the
 * paper's method: it exists to test that path.  MD_ERR_ARG for a null pruner. */
md_status md_pruner_set_wait(md_pruner *pruner, int32_t polls);

/* Allocation-free variant of md_eval_neighborhood + md_moves_read_leaders.  The paper has no
 * counterpart: it exists for callers that cannot call cudaMalloc (device memory budgeted up front,
 * latency-critical loops that must not enter the allocator, code handed only raw device buffers).
 * Evaluates operator ops_dev[s] (device int32 [n_sol]; a value outside [0, MD_N_OPS) skips the
 * solution, which then reads id 0, dF 0 and count 0) for every solution with its current lambda
 * and writes, to device buffers the caller owns, the leader id (0 when none) ids_dev [n_sol], its
 * dF dF_dev [n_sol] and the scored-move count n_scored_dev [n_sol].  No follower table and no
 * dump.  Scratch: a static device array of 1 MiB that every GPU loading the library holds until
 * exit; it must hold n_sol * (16 * 8 * min(ceil(n_customers * wpc / 8), 1024) + 8) bytes, with
 * wpc = min(max(floor(n_customers / 256), 1), 8), else MD_ERR_CAPACITY (for example 21 solutions
 * of 1000 customers fit: 48 008 bytes each).  The first call on each device looks up the array's device
 * address, so make that first call before any stream capture.  All calls share the array: calls
 * that overlap on the GPU (other streams, other threads) race and must be serialised by the
 * caller.  Calls no cudaMalloc or cudaFree. */
md_status md_eval_leaders_noalloc(md_solutions *sols, const int32_t *ops_dev, uint64_t *ids_dev,
                                  double *dF_dev, int64_t *n_scored_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MDLS_H */
