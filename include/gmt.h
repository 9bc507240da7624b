/*
 * gmt.h -- C ABI of the GB300 Group Marching Tree (GMT*) planner.
 *
 * The planner follows Ichter, Schmerling, Pavone, "Group Marching Tree:
 * Sampling-Based Approximately Optimal Motion Planning on GPUs" (2017).
 * Arguments follow the paper's problem statement (Problem 1, Section II: state
 * space X = [lo, hi], obstacle set X_obs, x_init, goal region X_goal, cost) and
 * the inputs of Algorithm 1 (n samples, connection radius r, group cost
 * threshold factor lambda).
 *
 * Conventions
 *  - Plain C: no CUDA, torch or C++ types.  A stream is passed as a
 *    `gmt_stream`, which is a cudaStream_t (NULL = the legacy default stream).
 *  - Memory: every array argument says whether it is HOST or DEVICE memory.
 *    The caller owns every array it passes in and every output array; the
 *    library owns the opaque handles (gmt_graph, gmt_batch, gmt_model,
 *    gmt_server) and the device memory inside them, released by *_free.
 *  - Errors: functions return a gmt_status; no C++ exception crosses the ABI.
 *    GMT_NO_PATH is a result, not an error (Problem 1: "report failure").
 *    gmt_last_error() returns a message for the last non-OK status of the
 *    calling host thread.
 *  - Device waits inside the kernels are bounded; a wait that runs out returns
 *    GMT_ERR_TIMEOUT and leaves the CUDA context usable.
 *  - There is no CPU fallback: every step of the path runs in the library's
 *    CUDA kernels.  Without a usable GPU, calls return GMT_ERR_CUDA.
 *  - Arithmetic: IEEE FP32 with round-to-nearest, no FMA contraction, IEEE
 *    division and square root in every decision, so results are reproducible.
 *  - Handles are not thread-safe: one handle must not be used by two calls
 *    at once (on any streams).
 */
#ifndef GMT_H
#define GMT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* gmt_stream;

typedef enum {
    GMT_OK = 0,
    GMT_NO_PATH = 1,          /* Alg. 1's failure outcome: V_open became empty */
    GMT_ERR_INVALID = -1,     /* bad argument, x_init in collision, sampling exhausted */
    GMT_ERR_OOM = -2,         /* device allocation failed or over the memory budget */
    GMT_ERR_CUDA = -3,        /* CUDA runtime error (message in gmt_last_error) */
    GMT_ERR_TIMEOUT = -4,     /* a bounded device wait ran out */
    GMT_ERR_ITER_LIMIT = -5,  /* more group expansions than gmt_params.max_iters */
    GMT_ERR_ADMISSION = -6    /* serving: request refused (no slot or memory) */
} gmt_status;

enum { GMT_COST_EUCLID = 0, GMT_COST_DI = 1, GMT_COST_DUBINS = 2 };
#define GMT_MAX_DIM 10

/* State space X = prod_a [lo[a], hi[a]] (Section II).
 * kind GMT_COST_EUCLID: geometric planning, cost = Euclidean arc length
 *   (Section II), dim in [2, GMT_MAX_DIM], pos_dim == dim.
 * kind GMT_COST_DI: 3D double integrator xdd = u (Section V-A), dim == 6,
 *   pos_dim == 3, state [p0 p1 p2 v0 v1 v2], cost = arrival time + integral of
 *   u^T u (the "mixed time/quadratic control effort" cost of Section V-A).
 * kind GMT_COST_DUBINS: Dubins airplane (Section V-A: a planar Dubins car of
 *   turning radius gmt_params.turn_radius with a single integrator in
 *   altitude), dim == 4, pos_dim == 3, state [x y z heading]; the trajectory
 *   is the shortest planar Dubins path with altitude linear in its arc length
 *   and the cost is its Euclidean length sqrt(L^2 + dz^2).  Pairs whose squared
 *   3D distance is at least (1 + 2^-6) r^2 are never connected (the cost is at
 *   least that distance).  An end turn of a word that computes within 2^-13
 *   rad of a full circle counts as the small negative turn it differs by. */
typedef struct {
    int32_t kind;
    int32_t dim;
    int32_t pos_dim;
    float lo[GMT_MAX_DIM];
    float hi[GMT_MAX_DIM];
} gmt_space;

/* X_obs: a union of `count` closed axis-aligned boxes in position space
 * (Section V-B).  lo and hi are DEVICE arrays [count][pos_dim], row-major,
 * owned by the caller; count == 0 allows NULL pointers. */
typedef struct {
    int32_t count;
    const float* lo;
    const float* hi;
} gmt_boxes;

/* X_goal: the closed ball |x - center| <= radius, over the position axes only
 * (pos_only != 0) or over the whole state (Problem 1). */
typedef struct {
    float center[GMT_MAX_DIM];
    float radius;
    int32_t pos_only;
} gmt_goal;

/* Alg. 1 inputs and implementation limits. */
typedef struct {
    int32_t n;            /* samples drawn by SampleFree(n); nodes N = n + 1 (node 0 = x_init) */
    float r;              /* connection radius; <= 0 selects Theorem 1's radius from eta, mu_free */
    float lambda;         /* group cost threshold factor, in [0, 1]; delta = fl(lambda*r);
                             0 = the FMT* limit (each group = the open nodes of minimum cost) */
    uint64_t seed;        /* Philox4x32-10 key of SampleFree */
    float seg_spacing;    /* geometric and Dubins airplane edges: a cost-c edge is checked at
                             max(2, ceil(c / seg_spacing) + 1) equally spaced points */
    int32_t traj_points;  /* double integrator edges: collision points along the trajectory (>= 2) */
    int32_t max_iters;    /* cap on group expansions; <= 0 means N + 1 */
    int32_t max_attempts; /* rejection-sampling attempts per node; <= 0 means 65536 */
    float eta;            /* Theorem 1 tuning parameter (>= 0), used when r <= 0 */
    float mu_free;        /* Lebesgue measure of X_free (upper bound), used when r <= 0 */
    int32_t spin_limit;   /* polls of a device-side wait before GMT_ERR_TIMEOUT; <= 0 = default */
    uint32_t debug_flags; /* GMT_DEBUG_*: test hooks, 0 in normal use */
    int32_t sampler;      /* GMT_SAMPLER_*: how SampleFree draws its n samples */
    float turn_radius;    /* GMT_COST_DUBINS: turning radius rho (> 0); such graphs
                             need r > 0 (Theorem 1's radius is for the geometric cost) */
} gmt_params;

/* SampleFree variants.
 *   GMT_SAMPLER_PHILOX: i.i.d. uniform samples (Philox4x32-10 keyed by seed);
 *     node 1 uniform in X_goal n X_free, nodes 2..n uniform in X_free, by
 *     rejection (max_attempts per node).
 *   GMT_SAMPLER_HALTON: the deterministic low-dispersion Halton sequence that
 *     the paper's experiments use (Sec. V): point k >= 1 has coordinate a equal
 *     to the radical inverse of k in the a-th prime base (2, 3, 5, 7, ...),
 *     mapped affinely onto X.  Node 1 is the first point mapped into the goal
 *     ball's bounding box (goal axes) that lies in X_goal n X_free; nodes 2..n
 *     are the points of X_free in the order of k.  seed is unused; at most
 *     max_attempts + 64 N points are tried per sequence (max_attempts <= 0:
 *     65536); r <= 0 selects gmt_connection_radius_halton. */
#define GMT_SAMPLER_PHILOX 0
#define GMT_SAMPLER_HALTON 1

/* Test hook: the plan kernel's inter-block barrier waits for one more arrival
 * than there are blocks, so every wait runs out and the call returns
 * GMT_ERR_TIMEOUT.  Used to test the bounded-wait path without a GPU fault. */
#define GMT_DEBUG_UNREACHABLE_BARRIER 0x1u
/* Test hooks for the neighbour build of 2D/3D geometric graphs, which picks
 * a cell list (candidates from the grid cells around each node) when the
 * radius is small against the domain and the all-pairs test otherwise; both
 * give the same CSR.  PAIRS_ALL forces the all-pairs test, PAIRS_CELLS the cell
 * list.  The cell list orders a row's columns with a bitmap of the row when
 * the graph has at most 32768 nodes, else by sorting a list of at most 1024
 * (a longer row falls back to the all-pairs test); CELLS_LIST forces the list
 * at any size. */
#define GMT_DEBUG_PAIRS_ALL 0x2u
#define GMT_DEBUG_PAIRS_CELLS 0x4u
#define GMT_DEBUG_CELLS_LIST 0x8u

typedef struct gmt_graph gmt_graph;

/* Read-only DEVICE views of a built graph (valid until the next build into, or
 * the release of, the handle).  Samples are SoA: coordinate a of node v is
 * X[a * x_pitch + v].  Out-rows list targets in ascending order; in-rows list
 * sources in ascending order.  For GMT_COST_EUCLID the cost is symmetric and
 * the in-arrays alias the out-arrays; the other kinds have their own in-CSR. */
typedef struct {
    int32_t kind, dim, pos_dim, N;
    int32_t x_pitch;
    int64_t E;
    float r;
    const float* X;          /* [dim][x_pitch] */
    const uint8_t* is_goal;  /* [N], 1 if the sample lies in X_goal */
    const int32_t* out_row;  /* [N+1] */
    const int32_t* out_col;  /* [E] */
    const float* out_cost;   /* [E] c(v, out_col[e]) */
    const int32_t* in_row;   /* [N+1] */
    const int32_t* in_col;   /* [E] */
    const float* in_cost;    /* [E] c(in_col[e], v) */
    const float* out_tau;    /* [E] double integrator: arrival time of the out-edge; NULL otherwise */
    const float* in_tau;     /* [E] double integrator: arrival time of the in-edge; NULL otherwise
                                (gmt_plan_static recomputes it when NULL) */
    float turn_radius;       /* Dubins airplane: the turning radius the costs were built with; 0 otherwise */
    const float* in_path;    /* [E][4] Dubins airplane: the in-edge's shortest planar word as (t, p, q, word),
                                word = LSL 0, RSR 1, LSR 2, RSL 3, RLR 4, LRL 5 stored as int32 bits;
                                NULL otherwise (gmt_plan_static recomputes it when NULL) */
} gmt_graph_view;

/* SampleFree and neighbour-set construction (Section III-B; the offline
 * precomputation of Section V-A).
 *   V = {x_init} U SampleFree(n): node 0 = x_init (HOST array [dim]), node 1 is
 *   drawn uniformly in X_goal n X_free, nodes 2..n uniformly in X_free.  Node k,
 *   attempt t uses Philox4x32-10 with counter (k, t, 0, block) and key (seed low
 *   32 bits, seed high 32 bits); coordinate a = lo[a] + u*(hi[a]-lo[a]) with
 *   u = (word >> 8) * 2^-24; the first attempt outside every box is kept.
 *   Edges: y -> x for y != x with c(y, x) < r (Section III-A), stored as CSR.
 * *graph: NULL to create a handle, or an existing handle whose device buffers
 * are reused (grown when needed).  space, boxes, goal, params: HOST structs
 * (box arrays inside are DEVICE).  Synchronises `stream` once (to size the
 * edge arrays).  Errors: GMT_ERR_INVALID (arguments; x_init outside X or in
 * X_obs; a node exhausted max_attempts), GMT_ERR_OOM, GMT_ERR_CUDA. */
gmt_status gmt_build_graph(const gmt_space* space, const gmt_boxes* boxes, const float* x_init,
                           const gmt_goal* goal, const gmt_params* params, gmt_graph** graph,
                           gmt_stream stream);

/* As gmt_build_graph, with `extra_count` caller samples appended after the
 * n + 1 SampleFree nodes (nodes n+1 .. n+extra_count), e.g. the learned
 * proposal's (gmt_propose).  extra: DEVICE [dim][extra_pitch].  Appended
 * samples must lie in X and outside X_obs (else GMT_ERR_INVALID).  Supported
 * for geometric dim <= 3 and the double integrator.  The radius is params->r
 * (or Theorem 1's for params->n when r <= 0). */
gmt_status gmt_build_graph_ex(const gmt_space* space, const gmt_boxes* boxes, const float* x_init,
                              const gmt_goal* goal, const gmt_params* params, const float* extra,
                              int32_t extra_count, int32_t extra_pitch, gmt_graph** graph, gmt_stream stream);

/* As gmt_build_graph, without the host synchronisation: when the handle's edge
 * arrays from earlier builds are at least as large as needed, the whole build
 * is only queued on `stream`, and its edge count and sampling status are read
 * by the next gmt_plan (or gmt_graph_get_view) on this handle, which returns
 * the errors gmt_build_graph would have returned.  If the edges do not fit
 * those arrays, that call rebuilds synchronously and the result is the same.
 * A new handle, the cell-list neighbour build or appended samples take the
 * synchronous path.  `boxes` (the struct's DEVICE arrays) must stay valid
 * until that plan or view. */
gmt_status gmt_build_graph_async(const gmt_space* space, const gmt_boxes* boxes, const float* x_init,
                                 const gmt_goal* goal, const gmt_params* params, gmt_graph** graph,
                                 gmt_stream stream);

gmt_status gmt_graph_get_view(const gmt_graph* graph, gmt_graph_view* view);
void gmt_graph_free(gmt_graph* graph);

/* Per-plan result and counters (host struct). */
typedef struct {
    int32_t status;       /* GMT_OK, GMT_NO_PATH or an error */
    int32_t goal_node;    /* minimum-cost tree node in X_goal (ties: lowest index), -1 if none */
    float path_cost;      /* cost[goal_node], +inf if none */
    int32_t path_len;     /* nodes on the path x_init .. goal_node, 0 if none */
    int64_t iters;        /* group expansions (non-empty groups G) */
    int64_t final_i;      /* threshold index i of the last expanded group */
    int64_t push_edges;   /* out-edges scanned from group nodes (Alg. 1's frontier push) */
    int64_t pull_edges;   /* in-edges scanned for parent selection (lazy parent) */
    int64_t checks;       /* lazy collision checks (Alg. 1) */
    int64_t failed;       /* checks that found a collision */
    int64_t tree_size;    /* nodes with finite cost at termination */
} gmt_plan_info;

/* Algorithm 1 on a built graph: one persistent kernel runs every wavefront
 * iteration (group selection, frontier push, lazy parent selection, one
 * collision check per candidate, set update, termination test) without host
 * round trips.  V_open in the lazy parent step is the open set at the start of the
 * iteration; a candidate whose check fails stays unexplored.
 *   boxes: obstacles for the collision checks (DEVICE arrays, may differ from
 *          the ones used at build time).
 *   parent, cost: DEVICE [N] outputs (parent -1 / cost +inf off the tree).
 *   path: DEVICE [N] output or NULL; receives x_init .. goal_node.
 *   info: HOST output.
 * Synchronises `stream`.  Returns info->status. */
gmt_status gmt_plan(gmt_graph* graph, const gmt_boxes* boxes, const gmt_params* params, int32_t* parent,
                    float* cost, int32_t* path, gmt_plan_info* info, gmt_stream stream);

/* Launch shape of gmt_plan on this graph (a tuning knob, not a semantic one:
 * every shape gives the same result).  cluster in [2, 16]: one thread-block
 * cluster of that many CTAs runs the plan with hardware cluster barriers
 * (blocks ignored); otherwise blocks == 1: one CTA with block barriers;
 * blocks > 1: a cooperative grid of that many CTAs (clamped to what can be
 * co-resident) with bounded software barriers; blocks == cluster == 0:
 * automatic (the largest cluster the GPU can hold, up to 16 CTAs).  threads:
 * CTA size, a multiple of 32 in [64, 1024], or 0 = automatic. */
gmt_status gmt_graph_set_launch(gmt_graph* graph, int32_t blocks, int32_t threads, int32_t cluster);

/* ---------------------------------------------------------------- batches
 * Many independent planning problems in one call (an extension of the paper's
 * single-query method: the same Algorithm 1 on every query).  Supported
 * queries: double integrator, Dubins airplane (turn_radius > 0, r > 0), and
 * geometric with dim 2 or 3. */
typedef struct {
    gmt_space space;
    gmt_boxes boxes;             /* DEVICE arrays, as for gmt_build_graph */
    float x_init[GMT_MAX_DIM];
    gmt_goal goal;
    gmt_params params;           /* r <= 0: Theorem 1 radius for this query's n and dim */
    /* Optional caller samples appended after the n + 1 SampleFree nodes, as
     * in gmt_build_graph_ex (nodes n+1 .. n+extra_count; each must lie in X
     * and outside X_obs, else the call fails with GMT_ERR_INVALID, or, on a
     * replay, that query's info.status is GMT_ERR_INVALID).  extra: DEVICE
     * [dim][extra_pitch], read on every call (also on replays), or NULL with
     * extra_count 0.  The radius stays Theorem 1's for params.n when r <= 0. */
    const float* extra;
    int32_t extra_count;
    int32_t extra_pitch;
} gmt_query;

typedef struct gmt_batch gmt_batch;

/* Samples, builds the neighbour CSR of, and plans every query.
 *   queries: HOST array [q].
 *   parent, cost: DEVICE outputs of sum_k N_k entries, N_k = n_k + 1 +
 *     extra_count_k; query k's nodes start at offset sum_{j<k} N_j.
 *   infos: HOST output [q].
 *   *batch: NULL to create a handle, or the handle of an earlier call, whose
 *     arena is reused.  If the queries (compared by value, including the box
 *     pointers) and the output pointers equal the previous call's, the whole
 *     device sequence is replayed from a CUDA graph captured on the first
 *     repeat (no host work between kernels); otherwise the batch is prepared
 *     anew (one host synchronisation to size the edge arrays).
 * Plan stage (see gmt_batch_set_mode): per (kind, dim) group, either one
 * persistent launch whose teams (one CTA or one cluster) take queries from a
 * device queue, largest edge count first, or one cooperative launch per 512
 * queries in which all queries advance one iteration per grid step.  Both
 * give every query the result of a single gmt_plan.  Synchronises `stream`.
 * Returns GMT_OK, or the first negative per-query status (all infos filled).
 * A query whose inputs changed in place so that its edge count outgrew the
 * replayed arena reports GMT_ERR_OOM in its info. */
gmt_status gmt_plan_batch(int32_t q, const gmt_query* queries, gmt_batch** batch, int32_t* parent, float* cost,
                          gmt_plan_info* infos, gmt_stream stream);

/* DEVICE views of query k's samples and CSR (and of its path, if `path` is
 * non-NULL) in the batch arena, valid until the next preparing call. */
gmt_status gmt_batch_get_view(const gmt_batch* batch, int32_t k, gmt_graph_view* view, int32_t** path);

/* Plan-stage scheme of a batch.
 *   GMT_BATCH_TEAMS: one persistent launch for every query of the batch; a
 *     team (a CTA or a cluster) runs one query at a time, one team barrier per
 *     Algorithm 1 iteration (double-buffered open-set snapshot; candidates
 *     are pulled from a team-wide queue as soon as they are claimed).  With
 *     one-CTA teams, when the largest query's wavefront state fits in a CTA's
 *     shared memory (about 36 bytes per node), each CTA keeps its query's
 *     whole state there (two barriers per iteration, every step but the CSR
 *     and sample reads on chip).
 *   GMT_BATCH_LOCKSTEP: one cooperative grid runs up to 512 queries at once,
 *     one Algorithm 1 iteration of every live query per grid step (two
 *     bounded grid barriers per step), so small groups of many queries fill
 *     the GPU together.
 *   GMT_BATCH_POOL: one persistent launch for every query of the batch (all
 *     kinds); each iteration of each query is split into work items (group
 *     selection over 32 open entries, the push of one group node, the lazy
 *     parent and check of one candidate) that any warp may take, so queries
 *     advance without team barriers and without waiting for one another.
 *   GMT_BATCH_AUTO: the autotuner's choice; before tuning, teams of 4 CTAs. */
typedef enum { GMT_BATCH_AUTO = 0, GMT_BATCH_TEAMS = 1, GMT_BATCH_LOCKSTEP = 2, GMT_BATCH_POOL = 3 } gmt_batch_mode;
gmt_status gmt_batch_set_mode(gmt_batch* batch, int32_t mode);

/* Launch shape of the batched plan stage: cluster = CTAs per team (teams
 * scheme only: 1, 2, 4, 8 or 16; 0 = tuned/automatic), threads per CTA (both
 * schemes; 0 = tuned/automatic). */
gmt_status gmt_batch_set_launch(gmt_batch* batch, int32_t cluster, int32_t threads);

/* The scheme and shape the next plan stage will use (outputs may be NULL);
 * cluster is 0 under the lockstep scheme. */
gmt_status gmt_batch_get_launch(const gmt_batch* batch, int32_t* mode, int32_t* cluster, int32_t* threads);

/* Autotuner: on a batch planned at least once, times the plan stage for every
 * team shape (cluster 1..16 x 256/512/1024 threads) and every lockstep shape
 * (256/512/1024 threads) on `stream`, keeps the fastest as the automatic
 * scheme and shape, and reports it (outputs may be NULL; best_cluster is 0
 * when lockstep wins, see gmt_batch_get_launch). */
gmt_status gmt_batch_autotune(gmt_batch* batch, gmt_stream stream, int32_t* best_cluster, int32_t* best_threads,
                              float* best_ms);

/* Device time of the plan stage (all plan launches, without the graph build)
 * of the last completed gmt_plan_batch or autotune call, in milliseconds. */
gmt_status gmt_batch_last_plan_ms(const gmt_batch* batch, float* ms);

void gmt_batch_free(gmt_batch* batch);

/* ---------------------------------------------------------------- replanning server
 * Continuous-batching request loop (an extension for planning inside a
 * control loop, Sec. V-C's setting): sessions keep samples and the neighbour
 * CSR resident (connection costs do not depend on the obstacles) plus a
 * per-edge cache of collision verdicts; each request brings the session's
 * current boxes, the cache entries of edges whose checked points' bounding box
 * meets the old or new place of a moved box are cleared, and the wavefront is
 * re-run (results identical to a fresh plan).  A worker thread admits queued
 * requests to free slots (CUDA streams with their own plan scratch) as soon as
 * they free up, so requests overlap on the device; a session has at most one
 * request running.  Sessions are admitted against a device-memory budget. */
typedef struct {
    int32_t slots;         /* concurrent requests (streams), >= 1 */
    int32_t cluster;       /* CTAs per plan: 0/1 = one CTA, 2..16 = a cluster */
    int32_t threads;       /* threads per CTA (0 = automatic) */
    int32_t max_nodes;     /* largest N of any session */
    int32_t max_boxes;     /* largest box count of any session */
    uint64_t memory_budget;/* bytes of device memory sessions may hold; 0 = what is free */
} gmt_server_config;

typedef struct {
    uint64_t request_id;
    int32_t session;
    int32_t status;        /* as gmt_plan_info.status */
    int32_t goal_node;
    float path_cost;
    int64_t iters;
    int64_t checks;        /* lazy checks (Alg. 1) */
    int64_t checks_computed; /* of those, not answered by the verdict cache */
    int64_t edges_checked; /* out-edges pushed + in-edges pulled */
    double queue_ms;       /* submit -> launch */
    double latency_ms;     /* submit -> plan finished on the device */
} gmt_server_result;

typedef struct gmt_server gmt_server;

gmt_status gmt_server_create(const gmt_server_config* config, gmt_server** server);
/* Stops the worker (after running requests finish) and frees everything. */
void gmt_server_free(gmt_server* server);
/* Builds a resident session: SampleFree + CSR for the problem (space, x_init,
 * goal, params as for gmt_build_graph) with `box_count` boxes given as HOST
 * arrays [box_count][pos_dim].  Spaces: double integrator, Dubins airplane,
 * geometric with dim 2 or 3 (else GMT_ERR_INVALID).  GMT_ERR_ADMISSION if its
 * estimated device memory does not fit the budget (or the free memory).
 * Synchronous. */
gmt_status gmt_server_open_session(gmt_server* server, const gmt_space* space, const float* x_init,
                                   const gmt_goal* goal, const gmt_params* params, int32_t box_count,
                                   const float* box_lo, const float* box_hi, int32_t* session);
/* Queues a replanning request for the session with its boxes now (HOST
 * arrays, same count as at open).  parent/cost: DEVICE [N] outputs or NULL
 * (they must stay valid until the result is polled).  Returns at once. */
gmt_status gmt_server_submit(gmt_server* server, int32_t session, uint64_t request_id, const float* box_lo,
                             const float* box_hi, int32_t* parent, float* cost);
/* Moves up to `max` finished results to `out` (HOST), waiting up to wait_ms
 * for the first one. */
gmt_status gmt_server_poll(gmt_server* server, gmt_server_result* out, int32_t max, int32_t* count,
                           int32_t wait_ms);
/* Waits for the session's requests, then frees it. */
gmt_status gmt_server_close_session(gmt_server* server, int32_t session);
/* The robot has moved: node 0 of the session becomes x_init (HOST [dim]).
 * Waits (up to 30 s, else GMT_ERR_TIMEOUT) for the requests submitted
 * before, then builds the session's graph again (same seed, the boxes of its
 * last request; node 0's rows are part of every other row's neighbours, so
 * the CSR is rebuilt rather than patched) with a cleared verdict cache;
 * requests submitted meanwhile wait and then plan on the new graph.
 * GMT_ERR_INVALID if x_init is outside X or inside one of those boxes; on any
 * error the session keeps its previous graph.  Synchronous. */
gmt_status gmt_server_move_start(gmt_server* server, int32_t session, const float* x_init);
gmt_status gmt_server_session_view(gmt_server* server, int32_t session, gmt_graph_view* view);

/* ---------------------------------------------------------------- learned proposal
 * An extension beyond the paper (which samples uniformly or with Halton
 * points): an MLP maps a G^3 voxel occupancy grid of the obstacles plus start
 * and goal to logits over C^3 coarse cells of the position space:
 *   H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Z = [H2, start, goal, 0],
 *   logits = Z W3^T + b3   (X [B, G^3], H1/H2 [B, hidden], Z [B, hidden+16]).
 * Forward and backward run on the tcgen05 BF16 GEMM (FP32 accumulation);
 * training minimises the softmax cross-entropy against a target distribution
 * over cells with AdamW on FP32 master weights. */
typedef struct {
    int32_t grid;       /* G: voxels per axis (32) */
    int32_t hidden;     /* hidden width (512), multiple of 64 */
    int32_t cells;      /* C: coarse cells per axis (16 -> 4096 logits) */
    int32_t max_batch;  /* largest batch of environments per call */
    uint64_t seed;      /* Philox key of the initial weights */
} gmt_model_config;

typedef struct gmt_model gmt_model;

/* DEVICE pointers into a model (parameters FP32 row-major [out][in], their
 * BF16 copies, the last gradients, logits [B][cells^3] and per-environment
 * losses of the last forward/backward).  The BF16 activations of the last
 * pass, row-major with one row per environment (valid for its first B rows):
 * H1, H2 [B][hidden] (after ReLU), Z [B][z_features] (H2, start, goal, zero
 * padding), and of the last backward dlog [B][cells^3] ((softmax - target)/B),
 * dH2, dH1 [B][hidden] (gradients after the ReLU masks). */
typedef struct {
    int32_t grid, hidden, cells, in_features, z_features, n_cells, max_batch;
    int64_t step;
    const float *W1, *b1, *W2, *b2, *W3, *b3;
    const float *gW1, *gb1, *gW2, *gb2, *gW3, *gb3;
    const void *W1_bf16, *W2_bf16, *W3_bf16;
    const float* logits;
    const float* loss;
    const void *H1, *H2, *Z, *dlog, *dH2, *dH1;
} gmt_model_view;

gmt_status gmt_model_create(const gmt_model_config* config, gmt_model** model);
void gmt_model_free(gmt_model* model);
gmt_status gmt_model_get_view(const gmt_model* model, gmt_model_view* view);

/* Voxel occupancy of B environments: voxel (i, j, k) of [0,1]^3 is 1 if its
 * centre ((i+.5)/G, (j+.5)/G, (k+.5)/G) lies in a box.  boxes: HOST array [B]
 * (box arrays DEVICE, 3D).  voxels: DEVICE BF16 [B][G^3], index (i G + j) G + k.
 * Synchronises `stream`. */
gmt_status gmt_voxelize(int32_t B, const gmt_boxes* boxes, int32_t grid, void* voxels, gmt_stream stream);

/* Forward pass.  voxels: DEVICE BF16 [B][G^3]; start_goal: DEVICE FP32 [B][6];
 * logits: DEVICE FP32 [B][C^3] or NULL (then read them through the view). */
gmt_status gmt_model_forward(gmt_model* model, int32_t B, const void* voxels, const float* start_goal,
                             float* logits, gmt_stream stream);
/* Forward + backward (gradients into the model, no update).  target: DEVICE
 * FP32 [B][C^3], rows summing to 1.  mean_loss: HOST, may be NULL. */
gmt_status gmt_model_backward(gmt_model* model, int32_t B, const void* voxels, const float* start_goal,
                              const float* target, float* mean_loss, gmt_stream stream);
/* Forward + backward + one AdamW step (beta 0.9/0.999, eps 1e-8; decay on the
 * weight matrices only).  Synchronises `stream`. */
gmt_status gmt_model_train_step(gmt_model* model, int32_t B, const void* voxels, const float* start_goal,
                                const float* target, float lr, float weight_decay, float* mean_loss,
                                gmt_stream stream);
/* Checkpoint: weights, Adam moments, step count and seed in one binary file. */
gmt_status gmt_model_save(const gmt_model* model, const char* path);
gmt_status gmt_model_load(gmt_model* model, const char* path);

/* Training target: histogram over C^3 cells of points every `spacing` along
 * the path (sample indices, DEVICE [len]) through samples X (DEVICE
 * [>=3][pitch], first three coordinates = position in [0,1]^3), plus eps in
 * every cell, normalised to sum 1.  hist: DEVICE FP32 [C^3]. */
gmt_status gmt_path_histogram(const float* X, int32_t pitch, const int32_t* path, int32_t len, int32_t cells,
                              float spacing, float eps, float* hist, gmt_stream stream);

/* Learned samples for one 3D geometric problem: one forward pass on the
 * voxelised boxes with start/goal (HOST [3] each), then `count` draws: a cell
 * from the softmax (inverse CDF), a uniform point inside it (Philox4x32-10,
 * counter (sample, attempt, 2, 0), key = seed), rejected while it lies in a
 * box.  samples: DEVICE [3][pitch].  Synchronises `stream`. */
gmt_status gmt_propose(gmt_model* model, const gmt_space* space, const gmt_boxes* boxes, const float* start,
                       const float* goal, int32_t count, uint64_t seed, float* samples, int32_t pitch,
                       gmt_stream stream);

/* gmt_propose for B problems at once: the voxelisation, one forward pass and
 * one sampling launch (one CTA per problem) per `max_batch` problems, and one
 * host synchronisation for the whole call.  Problem b draws `count` samples
 * exactly as gmt_propose would with seed seeds[b], from the logits of a
 * forward pass over its chunk of problems (the GEMMs' FP32 summation order
 * may depend on the chunk size, so a sample can differ from a single call's
 * where a draw lies within rounding of a cell boundary of the CDF).
 *   spaces, boxes: HOST arrays [B] (box arrays DEVICE, 3D geometric spaces).
 *   start_goal: HOST FP32 [B][6] (start xyz, goal xyz).
 *   seeds: HOST [B].
 *   samples: DEVICE FP32 [B][3][pitch], pitch >= count; problem b's rows
 *     start at samples + 3 b pitch (the layout gmt_query.extra takes).
 * Errors: GMT_ERR_INVALID (arguments; a sample exhausted its attempts). */
gmt_status gmt_propose_batch(gmt_model* model, int32_t B, const gmt_space* spaces, const gmt_boxes* boxes,
                             const float* start_goal, int32_t count, const uint64_t* seeds, float* samples,
                             int32_t pitch, gmt_stream stream);

/* ---------------------------------------------------------------- tensor cores
 * BF16 GEMM on the 5th-generation tensor cores (tcgen05, TMEM accumulator,
 * TMA loads), the building block of the learned sampling proposal:
 *   C[M, N] = A[M, K] . B[N, K]^T, FP32 accumulation.
 * A, B: DEVICE BF16 row-major, 16-byte aligned, K % 8 == 0.
 * epilogue 0: C (DEVICE FP32 [M, N]) = A.B^T;
 *          1: C_bf16 (DEVICE BF16 [M, N]) = bf16(relu(A.B^T + bias));
 *          2: C = A.B^T + bias.   bias: DEVICE FP32 [N] or NULL.
 * splits > 1 divides K among CTAs (split-K) and needs `workspace` (DEVICE FP32
 * [splits * M * N]); partial sums are reduced in a fixed order.
 * error_flag: DEVICE int, set to 1 if a bounded device wait ran out (the
 * output is then undefined); the caller zeroes it.  Asynchronous on `stream`. */
gmt_status gmt_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, const void* B, int32_t epilogue,
                         const float* bias, float* C, void* C_bf16, int32_t splits, float* workspace,
                         int32_t* error_flag, gmt_stream stream);

/* Allocation-free planning (an implementation entry point; the paper has no
 * counterpart).  Runs the same wavefront kernel as gmt_plan, for callers that
 * must not allocate device memory while they plan: a replanning loop inside a
 * control cycle (cudaMalloc/cudaFree can synchronise the device and have no
 * latency bound), or systems whose memory is fixed at start-up.
 *   space: HOST struct; its position bounds are used by double-integrator
 *          trajectory checks and must match the graph's kind and dimensions.
 *   graph: HOST struct of DEVICE arrays describing the neighbour CSR and the
 *          samples (layout as gmt_graph_view; e.g. from gmt_graph_get_view or
 *          the caller's own buffers).  graph->N <= GMT_STATIC_MAX_NODES, else
 *          GMT_ERR_INVALID.
 *   boxes, params, parent, cost, path, info, stream: as for gmt_plan.
 * The kernel's scratch is one fixed __device__ array inside the library
 * (about 2.6 MB on each GPU that loads it, held until the process exits); no
 * cudaMalloc, cudaFree or other allocating call is made.  The first call on a
 * device looks up that array's address and the plan kernel's largest resident
 * cluster; make it before any stream capture.  The launch shape is gmt_plan's
 * automatic one, but every check scans the boxes linearly (gmt_plan's box grid
 * for 128 or more boxes needs allocated scratch).
 * Every call on a device shares the array (its contents persist between calls;
 * each call clears the control block it needs), so calls that overlap on the
 * GPU race: serialise them.  Synchronises `stream`; returns info->status. */
#define GMT_STATIC_MAX_NODES 65536
gmt_status gmt_plan_static(const gmt_space* space, const gmt_graph_view* graph, const gmt_boxes* boxes,
                           const gmt_params* params, int32_t* parent, float* cost, int32_t* path,
                           gmt_plan_info* info, gmt_stream stream);

/* Per-kernel device times of the last gmt_build_graph / gmt_plan on a graph,
 * recorded with CUDA events on the caller's stream while profiling is on
 * (milliseconds; 0 for kernels that did not run).  Reading the profile waits
 * for the recorded events. */
typedef struct {
    float sample_ms;     /* SampleFree */
    float pair_ms;       /* all-pairs cost filter (neighbour bit matrix; for directed
                          * costs also its transpose, the in-edge bit matrix) */
    float transpose_ms;  /* 0: the pair filter writes the in-edge bit matrix (the field
                          * keeps the layout of earlier versions) */
    float scan_ms;       /* row offsets */
    float fill_ms;       /* CSR columns and costs */
    float plan_ms;       /* wavefront kernel */
    int32_t plan_blocks; /* launch shape used by the last plan (-k: a cluster of k CTAs) */
    int32_t plan_threads;
} gmt_profile;

/* enable: 0 off, 1 every stage (two events around each), 2 the plan kernel
 * only (events cost the device a few microseconds each). */
gmt_status gmt_graph_set_profiling(gmt_graph* graph, int32_t enable);
gmt_status gmt_graph_get_profile(gmt_graph* graph, gmt_profile* profile);

/* Theorem 1's radius r = 4 (1+eta)^(1/d) (1/d)^(1/d) (mu_free/zeta_d)^(1/d)
 * (log n / n)^(1/d), zeta_d the volume of the unit d-ball, evaluated in double
 * as 4 * pow((1+eta) * (1/d) * (mu_free/zeta_d) * (log(n)/n), 1/d). */
double gmt_connection_radius(int32_t n, int32_t d, double eta, double mu_free);

/* Radius for low-dispersion (Halton) samples.  Sec. III-B allows a smaller r
 * than Theorem 1's for such sequences without fixing one; this library's
 * reading drops Theorem 1's log n factor: 4 * pow((1+eta) * (1/d) *
 * (mu_free/zeta_d) * (1/n), 1/d). */
double gmt_connection_radius_halton(int32_t n, int32_t d, double eta, double mu_free);

/* Message for the last non-OK status returned to this host thread. */
const char* gmt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GMT_H */
