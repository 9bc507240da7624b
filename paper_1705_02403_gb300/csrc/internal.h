// Internal interfaces between the C-ABI layer (capi.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gmt.h"

namespace gmtk {

constexpr int kMaxDimHost = GMT_MAX_DIM;

// Problem description passed by value to the sampling and graph kernels.
struct SpaceArgs {
    int kind, d, dp;
    int N;        // nodes of the graph
    int n_sampled;  // nodes 0 .. n_sampled-1 are drawn by SampleFree; the rest are appended samples
    int pitch;    // row pitch of X and of the neighbour bit matrix (N rounded up to 32)
    float lo[kMaxDimHost], hi[kMaxDimHost];
    float x0[kMaxDimHost];
    float gc[kMaxDimHost];
    float grho;
    int gd;       // axes of the goal ball
    uint32_t key0, key1, stream;
    int max_attempts;
    float r;
    float r2_threshold;  // Euclidean: edge iff squared distance < r2_threshold (== sqrt(s) < r)
    float rho;           // Dubins airplane: turning radius
    int sampler;         // GMT_SAMPLER_PHILOX or GMT_SAMPLER_HALTON
    long long halton_cap;  // Halton points tried per sequence
};

struct BoxArgs {
    int count;
    const float* lo;
    const float* hi;
};

// Grid over the first two position axes for checks against many boxes: box b
// is listed in every cell its [lo, hi] overlaps on those axes (cells from
// cell(lo) to cell(hi), cell(x) = clamp(floor((x - lo_grid) * inv_h))), or, if
// that is more than kBoxGridMaxCells cells, in a list of big boxes.  A box
// that holds a point p is listed in p's cell: lo <= p <= hi gives
// cell(lo) <= cell(p) <= cell(hi), since every step of cell() is monotone in
// IEEE arithmetic.  A query tests the boxes of p's cell and the big boxes
// exactly, so its verdict equals testing every box.
struct BoxGridArgs {
    int use;            // 0: scan every box
    int g;              // cells per axis
    float lo[2], inv_h[2];
    const int* start;   // [g * g + 1] first list entry of each cell
    const int* list;    // box indices, grouped by cell
    const int* big;     // indices of the boxes over more than kBoxGridMaxCells cells
    const int* nbig;    // [1] their count
};
// Boxes from which the plan builds a grid (fewer are scanned directly).
constexpr int kBoxGridMinBoxes = 128;
// Cells a box may be listed in before it goes to the big-box list.
constexpr int kBoxGridMaxCells = 32;
// Cells per axis for `count` boxes.
inline int box_grid_cells(int count) {
    int g = 1;
    while (g < 64 && g * g < count) g *= 2;
    return g;
}
// Builds the grid: cnt [g*g] and nbig [1] must be zeroed; start [g*g + 1],
// list [count * kBoxGridMaxCells], big [count].
cudaError_t launch_box_grid(int dp, BoxArgs boxes, const BoxGridArgs& grid, int* cnt, int* start, int* list,
                            int* big, int* nbig, cudaStream_t st);

// Flags written by the sampling kernel.
enum { kSampleBadInit = 1, kSampleExhausted = 2, kSampleBadAppend = 4, kSampleTimeout = 8 };

// Halton SampleFree over several blocks: chunks of kHaltonChunk consecutive
// points, taken in order from a ticket; each publishes its count of free
// points, then (looking back over its predecessors) the running total, so its
// free points land at nodes 2 + total-before-it + rank, in the order of k.
constexpr int kHaltonChunk = 256;
// Scratch of the multi-block sampler: [0] ticket, [1] first chunk whose running
// total reaches the node count (INT_MAX before), then one 64-bit status word
// per chunk (8-byte aligned).  Zeroed, with [1] set high, before each launch.
inline size_t halton_scratch_bytes(long long cap) {
    return 16 + (size_t)((cap + kHaltonChunk - 1) / kHaltonChunk) * 8;
}

// sample.cu / graph.cu
// SampleFree with s.sampler's method (Halton: one block compacts the free
// points in order).
// grid: a box grid of `boxes` (use = 0 to scan them).
// scratch: halton_scratch_bytes(s.halton_cap) bytes prepared as described
// there (Halton sampler only; NULL runs the single-block sampler).
cudaError_t launch_sample(const SpaceArgs& s, BoxArgs boxes, const BoxGridArgs& grid, void* scratch, float* X,
                          uint8_t* is_goal,
                          int* flags, cudaStream_t st);
// maskT, in_count (double integrator and Dubins airplane; may be NULL): the
// same launch also writes the transposed bit matrix and the in-row counts (no
// transpose launch).
// tile_cnt (Euclidean graphs of 2 to 4 dimensions, may be NULL): receives,
// for launch_fill_tiles, the number of each row's edges in the tiles of
// kMaskWords mask words before each tile, [tile][pitch].
// elist, elist_n (double integrator, Dubins airplane; may be NULL): every
// edge is also listed as (row, column, cost bits, arrival-time bits or 0) at a
// slot counted by *elist_n (zero at launch; slots at or past elist_cap are
// not written), for launch_fill_list; a Dubins airplane list needs epath too
// (the edge's shortest word (t, p, q, word bits) at the same slot).
cudaError_t launch_pair_mask(const SpaceArgs& s, const float* X, uint32_t* mask, int* out_count,
                             uint32_t* maskT, int* in_count, cudaStream_t st, int* tile_cnt = nullptr,
                             int4* elist = nullptr, int* elist_n = nullptr, int elist_cap = 0,
                             float4* epath = nullptr);
// Does the tiled fill apply (Euclidean, 2 to 4 dimensions; on one graph from
// 4096 nodes, below which its extra prefix launch costs more than it saves;
// in a batch always, one launch serving every query), and how many tiles of
// mask words a row has.
inline bool fill_tiles_apply(int kind, int d, int N, bool batched) {
    return kind == GMT_COST_EUCLID && d >= 2 && d <= 4 && (batched || N >= 4096);
}
int fill_tiles_per_row(int N);
cudaError_t launch_scan(const int* count, int* row, int N, cudaStream_t st);
// Both directions' row offsets in one launch (count1 may be NULL: one scan).
// host_out (may be NULL; device-mapped host memory) receives flags[0],
// flags[1] and row0[N].  m0/pre0 and m1/pre1 (may be NULL): the same launch
// writes the word prefixes of those word-major bit matrices ([W][pitch] each:
// the set bits of a row's words before each word), for launch_fill_list.
cudaError_t launch_scan2(const int* count0, int* row0, const int* count1, int* row1, int N, const int* flags,
                         int* host_out, cudaStream_t st, const uint32_t* m0 = nullptr, int* pre0 = nullptr,
                         const uint32_t* m1 = nullptr, int* pre1 = nullptr, int pitch = 0);
// One CSR direction for the fill: the bit matrix rows come from (mask for
// out-rows, its transpose for in-rows), row offsets, and the outputs; tau
// (double integrator only, may be NULL) receives each edge's arrival time,
// path (Dubins airplane only, may be NULL) each edge's shortest word as
// (t, p, q, word bits) in 4 floats.
struct FillDir {
    const uint32_t* mask;
    const int* row;
    int* col;
    float* cost;
    float* tau;
    float* path;
    long long cap;  // > 0: the arrays hold `cap` edges; a larger edge count writes nothing
};
// Fills the out-CSR, and the in-CSR in the same launch when in.mask != NULL.
// ticket: one device int, zero at launch (the blocks' work counter).
cudaError_t launch_fill(const SpaceArgs& s, const float* X, const FillDir& out, const FillDir& in, int* ticket,
                        cudaStream_t st);
// Double integrator, Dubins airplane: both CSRs from the edge list of
// launch_pair_mask (list_cap slots; epath: the Dubins words, NULL for the
// double integrator) and the word prefixes of launch_scan2 (pre_out for
// out.mask, pre_in for in.mask), with no cost evaluated again.  Writes nothing
// if the edge count exceeds out.cap (> 0) or list_cap.
cudaError_t launch_fill_list(const SpaceArgs& s, const int4* elist, const float4* epath, int list_cap,
                             const FillDir& out, const FillDir& in, const int* pre_out, const int* pre_in,
                             cudaStream_t st);
// The out-CSR of a Euclidean graph of 2 to 4 dimensions from the mask and the
// per-tile prefixes of launch_pair_mask: one block per mask tile, columns
// staged in shared memory.  Reads its inputs only, so it may run again.  A
// graph whose edge count exceeds out.cap (> 0) writes nothing.
cudaError_t launch_fill_tiles(const SpaceArgs& s, const float* X, const FillDir& out, int* tile_cnt,
                              cudaStream_t st);

// Cell-list neighbour search (geometric graphs, 2 or 3 dimensions): a uniform
// grid over the position bounds whose cell side h is at least 1.01 r, so a
// pair closer than r by the FP32 edge predicate lies in the same or adjacent
// cells on every axis however the cell coordinates round (with at most 2^16
// cells, the rounding of (x - lo) / h stays below 10^-4 cell, against a 1%
// margin).  Cell index: ((c2 g1) + c1) g0 + c0.
struct CellGrid {
    int g[3];      // cells per axis (1 on unused axes)
    float lo[3];
    float inv_h;   // 1 / h
    int ncells;
    int list_only;  // the fill sorts a list even where a bitmap would fit (test hook)
};
// Shared-memory words per warp of the cell-list fill: a bitmap of the row's
// columns for graphs of at most 32 kCellList nodes, else a list of at most
// kCellList neighbours to sort (a longer row falls back to the all-pairs
// build).  cell_fill_fits says whether a longest row of max_deg fits.
__host__ __device__ inline bool cell_fill_fits(const CellGrid& cg, int N, int max_deg) {
    return (!cg.list_only && (N + 31) / 32 <= 1024) || max_deg <= 1024;
}
constexpr int kCellList = 1024;
// Returns false when the cell list does not apply (not a 2D/3D geometric
// graph); *pays is false when the 3^d cells around a node would hold more than
// a quarter of the domain.
bool make_cell_grid(int kind, int d, const float* lo, const float* hi, float r, int N, bool batched, CellGrid* cg,
                    bool* pays);
cudaError_t launch_cells_count(const SpaceArgs& s, const float* X, const CellGrid& cg, int* cell_of, int* cell_cnt,
                               cudaStream_t st);
// cell_cnt returns to zero.
cudaError_t launch_cells_scatter(int N, const int* cell_of, const int* cell_start, int* cell_cnt, int* sorted,
                                 cudaStream_t st);
// fill = false: out_count[v] = neighbours of v, max_deg = their maximum; fill
// = true: columns (ascending) and costs of every row at row[v]; a row longer
// than kCellList sets *overflow and writes nothing.
cudaError_t launch_cells_rows(const SpaceArgs& s, const float* X, const CellGrid& cg, const int* cell_of,
                              const int* cell_start, const int* sorted, bool fill, int* out_count, int* max_deg,
                              const int* row, int* col, float* cost, int* overflow, cudaStream_t st);

// Workspace and control block of one plan (all device memory).  Counters are
// double-buffered by iteration parity.  Open list j holds its kept entries in
// [0, kept) and the nodes opened by the previous iteration in
// [M - new_count[j], M) (M: the list's capacity).  gk[j] packs two counters
// that grow in the same phase, so one atomic reserves both: the low half
// counts group list j, the high half the kept entries of open list j ^ 1.
// The lockstep kernel keeps a query's whole open count in open_count and its
// minimum open cost in min_keep.
struct PlanCtl {
    unsigned bar_count, bar_gen;
    int error;
    int status;
    unsigned long long gk[2];
    int new_count[2];
    int cand_count[2];   // candidates claimed in an iteration of parity j
    int open_count[2];
    unsigned min_keep[2];  // minimum cost (as bits) over the kept entries
    unsigned min_new[2];   // ... over the newly opened nodes
    int goal_flag[2];    // the group held a goal node
    int iters;
    int final_i;
    int goal_node;
    int path_len;
    unsigned long long goal_key;
    unsigned long long push_edges, pull_edges, checks, failed, tree_size;
    unsigned long long checks_computed;  // checks not answered by the verdict cache
    // The one-barrier wavefront (plan_fused.cuh) keeps its per-iteration
    // counters in three sets (iteration i uses set i % 3): group entries (low
    // half) and kept entries (high half), nodes opened, minimum kept and
    // opened cost (as bits), group held a goal node.
    unsigned long long gk3[3];
    int new3[3];
    unsigned min_keep3[3], min_new3[3];
    int goal3[3];
    // ... and its candidate queue, by parity: cand_count[j] reserves entries,
    // ticket[j] deals them out, pushed[j] counts the warps done pushing.
    int ticket[2];
    unsigned pushed[2];
};

struct PlanArgs {
    int kind, d, dp, N, pitch;
    const float* X;
    const uint8_t* is_goal;
    const int* out_row;
    const int* out_col;
    const int* in_row;
    const int* in_col;
    const float* in_cost;
    const float* in_tau;  // double integrator: arrival time per in-edge (NULL: recompute)
    const float* in_path; // Dubins airplane: (t, p, q, word bits) per in-edge (NULL: recompute)
    BoxArgs boxes;
    BoxGridArgs grid;  // use = 0 unless the plan built one
    float pos_lo[3], pos_hi[3];
    float r, delta, seg_spacing;
    float rho;            // Dubins airplane: turning radius
    int traj_points, max_iters, spin_limit;
    unsigned debug_flags;
    float* cost;
    int* parent;
    int* path;
    float* ocost;         // open-set snapshot (cost if open, +inf otherwise)
    int* stamp;
    int* list_g[2];
    int2* list_open[2];   // (node, cost bits) of each open node; N entries each
    int* list_cand;
    PlanCtl* ctl;
    // Optional device-mapped host copy of the control block: the plan kernel
    // writes the final control block there once the plan is over, so the
    // caller needs no device-to-host copy (NULL: not written).
    PlanCtl* host_ctl;
    // Optional per-edge verdict cache (in-CSR order): 0 unknown, 1 free,
    // 2 collides.  A known verdict answers the check; an unknown one is
    // computed and stored.  Valid only while the obstacles that could change
    // the verdict stay where they were (the serving loop clears the entries
    // that moved boxes touch before every plan).
    uint8_t* verdict;
    // Set by the batched path: the CSR may only be read if the edge count the
    // build produced fits the slice that was filled (else GMT_ERR_OOM).
    int check_edges;
    long long edge_cap;
};

// Plan list scratch: open x2 (int2 entries) first, so both stay 8-byte
// aligned for any M when `base` is; then G x2 and the candidates (ints).
constexpr int kPlanListInts = 7;
__host__ __device__ inline size_t plan_list_stride(size_t M) { return (kPlanListInts * M + 3) / 4 * 4; }
__host__ __device__ inline void assign_plan_lists(PlanArgs& a, int* base, size_t M) {
    a.list_open[0] = (int2*)base;
    a.list_open[1] = (int2*)(base + 2 * M);
    a.list_g[0] = base + 4 * M;
    a.list_g[1] = base + 5 * M;
    a.list_cand = base + 6 * M;
}

// Largest box count staged in shared memory (2 * count * DP floats).
__host__ __device__ constexpr int smem_box_cap(int dp) { return 4096 / dp; }
// Dynamic shared memory of a plan launch: the staged boxes, or, when it is
// larger and fits within 48 KB beside the kernel's own static shared memory
// (at most kPlanStaticSmem bytes), the parent array of N nodes (read for the
// path walk once the wavefront is over).
constexpr size_t kPlanStaticSmem = 512;
inline size_t plan_smem_bytes(int staged_boxes, int dp, int N) {
    const size_t boxes = (size_t)2 * staged_boxes * dp * sizeof(float);
    const size_t parents = (size_t)N * sizeof(int);
    return parents + kPlanStaticSmem <= 48 * 1024 && parents > boxes ? parents : boxes;
}

// Per-team scratch of the batched wavefront: team t uses the slices
// [2 t max_nodes, 2 (t+1) max_nodes) of ocost (two snapshot buffers),
// [t max_nodes, (t+1) max_nodes) of stamp and
// [t plan_list_stride(max_nodes), (t+1) plan_list_stride(max_nodes)) of lists.
struct BatchScratch {
    float* ocost;
    int* stamp;
    int* lists;
    int max_nodes;
};

// Lockstep batched wavefront (plan_multi.cu).  At most kLockMaxQueries
// queries per launch; every block queues up to kLockQueue candidates per
// super-iteration in shared memory (further claims are pulled at once by the
// warp that made them).
constexpr int kLockMaxQueries = 512;
constexpr int kLockQueue = 1024;

// Grid-wide counters of one lockstep launch (zeroed by the caller).  Open
// list j holds its kept entries in [0, keep) and its newly opened ones in
// [nodes - new_total[j], nodes).  gk[j] packs two counters that grow in the
// same phase: the low half counts group list j, the high half the kept
// entries of open list j ^ 1.
struct LockCtl {
    PlanCtl team;  // barrier and error flag
    unsigned long long gk[2];
    int new_total[2];
};

struct LockScratch {
    LockCtl* ctl;
    int4* open[2];    // (node, cost bits, query, 0); `nodes` entries each
    int2* glist[2];   // (query, node); `nodes` entries each
    float* ocost;     // open-snapshot cost of every node of every query
    int* stamp;       // claim stamp of every node (INT_MAX: in the tree)
    const int* base;  // nq + 1 node offsets: query k owns [base[k], base[k+1])
    int nodes;        // base[nq]
};

// Pool scheme of the batched wavefront (plan_pool.cu): per-query scheduling
// state.  The claim word packs the current stage, its item count and the
// items claimed; done counts the stage's completed items.  The iteration
// fields are written before the stage that reads them is published.  A
// query's PlanArgs.ocost holds 2 N floats (the two snapshot buffers).
struct PoolIter {
    int it;        // iterations begun (the parity of the current one is it & 1)
    int ncur;      // entries of the open list
    int nk;        // of those, kept entries at its front (the rest at its back)
    int ng_prev;   // nodes of the previous group
    float theta;   // group threshold of this iteration
    int ng;        // nodes of this iteration's group (PUSH stage)
    long long i;   // threshold index
    int nc;        // candidates of this iteration (PULL stage)
    int pad;
};
struct __align__(64) PoolQ {
    unsigned long long word;
    int done;
    int live;
    PoolIter iter;
};
static_assert(sizeof(PoolQ) == 64, "one PoolQ per 64-byte line");
struct PoolCtl {
    int finished;  // queries done
    int error;     // GMT_ERR_TIMEOUT if a bounded wait ran out
};
// Runs the queries args[order[0 .. nq)] (largest first) in one persistent
// launch of `blocks` x `threads` (after a per-query initialisation launch).
// ecum: nq + 1 running sums of the queries' edge counts in that order (warps
// are dealt to queries in proportion); qs: nq entries; pool: zeroed before the
// call.  all_kinds = false: every query is geometric (a kernel with fewer
// registers).
cudaError_t launch_plan_pool(const PlanArgs* args, const int* order, const long long* ecum, int nq, PoolQ* qs,
                             PoolCtl* pool, bool all_kinds, int blocks, int threads, cudaStream_t st);
// Co-resident blocks of the pool kernel with `threads` threads (0 if none).
int plan_pool_max_blocks(int threads, bool all_kinds);

// mlp.cu: C = A . B^T on the tensor cores (BF16 in, FP32 accumulate);
// epilogue 0 = FP32 store, 1 = BF16 relu(x + bias), 2 = FP32 x + bias.
cudaError_t gemm_bf16_tn(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* B, int epilogue,
                         const float* bias, float* C, __nv_bfloat16* Cb, int ldc, int splits, float* partial,
                         int* error, cudaStream_t st);

// graph.cu: copies `count` appended samples (DEVICE [d][src_pitch]) into X
// columns first.. and computes their goal flags; sets flags kSampleBadAppend
// for a sample outside X or inside a box.
cudaError_t launch_append(const SpaceArgs& s, BoxArgs boxes, const float* src, int src_pitch, int first, int count,
                          float* X, uint8_t* is_goal, int* flags, cudaStream_t st);

// capi.cu: sets the message returned by gmt_last_error() on this host thread.
void record_error(const char* msg);

// plan.cu
// Launches the wavefront for one plan.  cluster > 1: one thread-block cluster
// of that many CTAs with hardware cluster barriers; else blocks <= 1: a single
// CTA with block barriers; else a cooperative grid of `blocks` CTAs that
// synchronises through bounded global barriers.
cudaError_t launch_plan(const PlanArgs& a, int blocks, int threads, cudaStream_t st, int cluster = 0);
int plan_max_coresident_blocks(int kind, int dp, int threads);
int plan_max_cluster(int kind, int dp, int threads);
// Persistent batched wavefront (one barrier per iteration) over the `nq`
// queries queries[order[0 .. nq)] of any kinds, taken in that order from the
// device counter `next` (zeroed by the caller); `slot` holds one int per team.
// cluster <= 1: teams are single CTAs, which keep the whole wavefront state
// in shared memory when the largest query (max_n nodes) fits
// (batch_state_fits; no scratch used), else use the scratch.  smem: dynamic
// shared memory per CTA (the largest plan_smem_bytes of the queries).
// all_kinds = false: every query is geometric (a kernel with fewer
// registers).  plan_batch_max_teams: resident teams of a shape; with
// smem_state = false, of the scratch-using kernels only (for sizing the
// scratch).
cudaError_t launch_plan_batch(const PlanArgs* queries, const int* order, int nq, int* next, int* slot,
                              const BatchScratch& scratch, int teams, int threads, int cluster, size_t smem,
                              int max_n, bool all_kinds, cudaStream_t st);
int plan_batch_max_teams(int threads, int cluster, size_t smem, int max_n, bool smem_state, bool all_kinds);
bool batch_state_fits(size_t smem, int max_n);
// plan_multi.cu: one cooperative grid of `blocks` CTAs advances all `nq`
// queries of one (kind, dp) group together (nq <= kLockMaxQueries).  The
// queries' PlanCtl blocks must be zeroed before the launch.
cudaError_t launch_plan_lockstep(int kind, int dp, const PlanArgs* queries, int nq, const LockScratch& s, int blocks,
                                 int threads, cudaStream_t st);
int plan_lockstep_max_blocks(int kind, int dp, int threads);

}  // namespace gmtk
