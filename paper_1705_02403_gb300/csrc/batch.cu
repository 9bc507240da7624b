// Batched planning (gmt_plan_batch): hundreds of independent queries of uneven
// size, each with its own samples, obstacles, radius and seed, run through the
// same kernels as single plans.
//
// Queries are grouped by (cost kind, position dimension) so that each group
// runs one instantiation of every kernel.  The build kernels cover all queries
// of a group in one launch: every block (or warp, or thread) finds its query
// by binary search over per-query prefix offsets of the work units.  The plan
// stage is one persistent launch per group in which teams (a CTA or a cluster)
// take queries from a device queue, largest first.  When the same batch is
// planned again (same descriptors, same outputs), the whole device sequence is
// replayed from a CUDA graph captured on the previous call.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "cells_body.cuh"

namespace gmtk {

struct QueryDev {
    SpaceArgs s;
    BoxArgs boxes;
    float* X;
    uint8_t* is_goal;
    int* flags;
    uint32_t* mask;
    uint32_t* maskT;
    int* out_count;
    int* in_count;
    int* out_row;
    int* in_row;
    int* out_col;
    float* out_cost;
    float* out_tau;
    int* in_col;
    float* in_cost;
    float* in_tau;
    float* in_path;  // Dubins airplane: (t, p, q, word) per in-edge, 16-byte aligned
    long long edge_cap;
    // cell-list neighbour build (2D/3D geometric queries with a small radius)
    CellGrid cg;
    int use_cells;
    int* cell_of;
    int* cell_sorted;
    int* cell_cnt;
    int* cell_start;
    int* cell_info;  // [longest row, a row overflowed the fill's list]
    // caller samples appended after the n_sampled SampleFree nodes
    const float* extra;
    int extra_pitch;
    // tiled fill (all-pairs Euclidean queries): per-tile row counts [tile][pitch]
    int* tile_cnt;
};

// index k with off[k] <= t < off[k+1] (off has nq+1 entries, off[0] = 0)
__device__ __forceinline__ int find_query(const long long* __restrict__ off, int nq, long long t) {
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// SampleFree of a group's nodes, one thread per node (any queries): the
// draws of sample_node, with the box test of an attempt taken over every box
// without early exit (one uniform loop per warp instead of lanes leaving it at
// different boxes).  Each node's sample is sample_node's.
template <int D, int DP>
__global__ void __launch_bounds__(128) batch_sample_kernel(const QueryDev* __restrict__ Q,
                                                           const long long* __restrict__ off, int nq) {
    const long long tn = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tn >= off[nq]) return;
    const int k = find_query(off, nq, tn);
    const QueryDev& q = Q[k];
    const int v = (int)(tn - off[k]);
    if (v >= q.s.n_sampled) {  // an appended sample
        append_node<D, DP>(q.s, q.boxes, q.extra, q.extra_pitch, q.s.n_sampled, q.X, q.is_goal, q.flags,
                           v - q.s.n_sampled);
        return;
    }
    if (q.s.sampler == GMT_SAMPLER_HALTON) return;  // batch_halton_kernel
    const BoxGridArgs no_grid{};
    if (v == 0) {
        sample_node<D, DP>(q.s, q.boxes, no_grid, q.X, q.is_goal, q.flags, 0);
        return;
    }
    float x[D];
    bool ok = false;
    for (int t = 0; t < q.s.max_attempts && !ok; ++t) ok = sample_attempt<D, DP, true>(q.s, q.boxes, no_grid, v, t, x);
    if (!ok) atomicOr(q.flags, kSampleExhausted);
#pragma unroll
    for (int a = 0; a < D; ++a) q.X[(size_t)a * q.s.pitch + v] = x[a];
    q.is_goal[v] = in_goal_ball(x, q.s.gd, q.s.gc, q.s.grho) ? 1 : 0;
}

// One block per query of the group; queries that sample with Philox return.
template <int D, int DP>
__global__ void __launch_bounds__(kHaltonThreads) batch_halton_kernel(const QueryDev* __restrict__ Q) {
    const QueryDev& q = Q[blockIdx.x];
    if (q.s.sampler != GMT_SAMPLER_HALTON) return;
    const BoxGridArgs no_grid{};
    halton_sample_block<D, DP>(q.s, q.boxes, no_grid, q.X, q.is_goal, q.flags);
}

template <int KIND, int D>
__global__ void __launch_bounds__(kMaskRows) batch_mask_kernel(const QueryDev* __restrict__ Q,
                                                               const long long* __restrict__ off, int nq) {
    const long long b = blockIdx.x;
    const int k = find_query(off, nq, b);
    const QueryDev& q = Q[k];
    const int rb = (q.s.N + kMaskRows - 1) / kMaskRows;
    const int t = (int)(b - off[k]);
    mask_tile<KIND, D>(q.s, q.X, q.mask, q.out_count, t % rb, t / rb, q.tile_cnt);
}

__global__ void __launch_bounds__(kDIRows, 8) batch_mask_di_kernel(const QueryDev* __restrict__ Q,
                                                               const long long* __restrict__ off, int nq) {
    const long long b = blockIdx.x;
    const int k = find_query(off, nq, b);
    const QueryDev& q = Q[k];
    const int rb = (q.s.N + kDIRows - 1) / kDIRows;
    const int t = (int)(b - off[k]);
    mask_di_tile(q.s, q.X, q.mask, q.out_count, t % rb, t / rb);
}

__global__ void __launch_bounds__(kDubRows) batch_mask_dubins_kernel(const QueryDev* __restrict__ Q,
                                                                    const long long* __restrict__ off, int nq) {
    const long long b = blockIdx.x;
    const int k = find_query(off, nq, b);
    const QueryDev& q = Q[k];
    const int rb = (q.s.N + kDubRows - 1) / kDubRows;
    const int t = (int)(b - off[k]);
    mask_dubins_tile(q.s, q.X, q.mask, q.out_count, t % rb, t / rb);
}

__global__ void __launch_bounds__(256) batch_transpose_kernel(const QueryDev* __restrict__ Q,
                                                              const long long* __restrict__ off, int nq) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (w >= off[nq]) return;
    const int k = find_query(off, nq, w);
    const QueryDev& q = Q[k];
    transpose_task(q.s.N, q.s.pitch, q.mask, q.maskT, q.in_count, w - off[k]);
}

__global__ void __launch_bounds__(1024) batch_scan_kernel(const QueryDev* __restrict__ Q, int incoming) {
    const QueryDev& q = Q[blockIdx.x];
    if (incoming) scan_rows(q.in_count, q.in_row, q.s.N);
    else scan_rows(q.out_count, q.out_row, q.s.N);
}

// ---- cell-list neighbour build (queries with use_cells; the others return)
template <int D>
__global__ void __launch_bounds__(256) batch_cells_count_kernel(const QueryDev* __restrict__ Q,
                                                                const long long* __restrict__ off, int nq) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= off[nq]) return;
    const int k = find_query(off, nq, t);
    const QueryDev& q = Q[k];
    if (q.use_cells) cell_count_node<D>(q.s, q.X, q.cg, q.cell_of, q.cell_cnt, (int)(t - off[k]));
}

__global__ void __launch_bounds__(1024) batch_cells_scan_kernel(const QueryDev* __restrict__ Q) {
    const QueryDev& q = Q[blockIdx.x];
    if (q.use_cells) scan_rows(q.cell_cnt, q.cell_start, q.cg.ncells);
}

__global__ void __launch_bounds__(256) batch_cells_scatter_kernel(const QueryDev* __restrict__ Q,
                                                                  const long long* __restrict__ off, int nq) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= off[nq]) return;
    const int k = find_query(off, nq, t);
    const QueryDev& q = Q[k];
    if (q.use_cells) cell_scatter_node(q.s.N, q.cell_of, q.cell_start, q.cell_cnt, q.cell_sorted, (int)(t - off[k]));
}

// One CTA per (query, cell) of the cell-list queries (off: cumulative cell
// counts, 0 for the other queries).  Fill pass: a query whose longest row
// outgrew the sort list (only possible if a replayed batch's inputs changed in
// place) gets an edge count its plan rejects (GMT_ERR_OOM); so does one whose
// edge count outgrew its slice.
template <int D, bool FILL>
__global__ void __launch_bounds__(kCellWarps * 32) batch_cells_tile_kernel(const QueryDev* __restrict__ Q,
                                                                           const long long* __restrict__ off, int nq,
                                                                           int words) {
    extern __shared__ int cell_buf[];
    const long long c = blockIdx.x;
    if (c >= off[nq]) return;
    const int k = find_query(off, nq, c);
    const QueryDev& q = Q[k];
    if (!q.use_cells) return;
    if (FILL && (long long)q.out_row[q.s.N] > q.edge_cap) return;
    cell_tile<D, FILL>(q.s, q.X, q.cg, q.cell_start, q.cell_sorted, q.out_count, q.cell_info, q.out_row, q.out_col,
                       q.out_cost, q.cell_info + 1, cell_buf, words, (int)(c - off[k]));
    if (FILL && threadIdx.x == 0 && __ldcg(&q.cell_info[1]) != 0) q.out_row[q.s.N] = INT_MAX;
}

// One warp per (query, row).  A query whose edge count exceeds the slice it was
// given (only possible if a replayed batch's inputs changed in place) writes
// nothing; its plan then reports GMT_ERR_OOM.
template <int KIND, int D>
__global__ void __launch_bounds__(kFillWarps * 32) batch_fill_kernel(const QueryDev* __restrict__ Q,
                                                                     const long long* __restrict__ off, int nq) {
    __shared__ int list[kFillWarps][kFillList];
    const long long w = (long long)blockIdx.x * kFillWarps + (threadIdx.x >> 5);
    if (w >= off[nq]) return;
    const int k = find_query(off, nq, w);
    const QueryDev& q = Q[k];
    if (q.use_cells || q.tile_cnt) return;
    const bool incoming = blockIdx.y == 1;  // in-rows (double integrator, Dubins airplane)
    const int* row = incoming ? q.in_row : q.out_row;
    if ((long long)row[q.s.N] > q.edge_cap) return;
    if (incoming)
        fill_row<KIND, D, true>(q.s, q.X, q.maskT, q.in_row, q.in_col, q.in_cost, q.in_tau, q.in_path,
                                (int)(w - off[k]), list[threadIdx.x >> 5]);
    else
        fill_row<KIND, D, false>(q.s, q.X, q.mask, q.out_row, q.out_col, q.out_cost, q.out_tau, nullptr,
                                 (int)(w - off[k]), list[threadIdx.x >> 5]);
}

// Tiled fill of the all-pairs Euclidean queries: after the pair filter, the
// per-tile counts become prefixes (one thread per row; off: cumulative node
// counts); the fill, one block per mask tile (off: cumulative mask tiles),
// then only reads them, so the build's back half can run again (the
// autotuner does).  A query whose edge count exceeds its slice writes
// nothing; its plan then reports GMT_ERR_OOM.
__global__ void __launch_bounds__(256) batch_tile_prefix_kernel(const QueryDev* __restrict__ Q,
                                                                const long long* __restrict__ off, int nq) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= off[nq]) return;
    const int k = find_query(off, nq, t);
    const QueryDev& q = Q[k];
    if (!q.tile_cnt) return;
    const int W = (q.s.N + 31) / 32;
    tile_prefix_row(q.tile_cnt, q.s.pitch, (W + kMaskWords - 1) / kMaskWords, (int)(t - off[k]));
}

template <int D>
__global__ void __launch_bounds__(kMaskRows) batch_fill_tile_kernel(const QueryDev* __restrict__ Q,
                                                                    const long long* __restrict__ off, int nq) {
    const long long b = blockIdx.x;
    const int k = find_query(off, nq, b);
    const QueryDev& q = Q[k];
    if (!q.tile_cnt || (long long)q.out_row[q.s.N] > q.edge_cap) return;
    const int rb = (q.s.N + kMaskRows - 1) / kMaskRows;
    const int t = (int)(b - off[k]);
    fill_tile_euclid<D>(q.s, q.X, q.mask, q.out_row, q.tile_cnt, q.out_col, q.out_cost, t % rb, t / rb);
}

namespace {
template <int D, int DP>
void sample_g(const QueryDev* Q, const long long* off, int nq, long long total, bool halton, cudaStream_t st) {
    batch_sample_kernel<D, DP><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(Q, off, nq);
    if (halton) batch_halton_kernel<D, DP><<<nq, kHaltonThreads, 0, st>>>(Q);
}
template <int KIND, int D>
void mask_g(const QueryDev* Q, const long long* off, int nq, long long tiles, cudaStream_t st) {
    if (KIND == GMT_COST_DI) batch_mask_di_kernel<<<(unsigned)tiles, kDIRows, 0, st>>>(Q, off, nq);
    else if (KIND == GMT_COST_DUBINS) batch_mask_dubins_kernel<<<(unsigned)tiles, kDubRows, 0, st>>>(Q, off, nq);
    else batch_mask_kernel<KIND, D><<<(unsigned)tiles, kMaskRows, 0, st>>>(Q, off, nq);
}
template <int KIND, int D>
void fill_g(const QueryDev* Q, const long long* off, int nq, long long rows, cudaStream_t st) {
    const dim3 grid((unsigned)((rows + kFillWarps - 1) / kFillWarps), KIND == GMT_COST_EUCLID ? 1 : 2);
    batch_fill_kernel<KIND, D><<<grid, kFillWarps * 32, 0, st>>>(Q, off, nq);
}
}  // namespace

cudaError_t batch_sample(int kind, int d, const QueryDev* Q, const long long* off, int nq, long long total,
                         bool halton, cudaStream_t st) {
    if (kind == GMT_COST_DI) sample_g<6, 3>(Q, off, nq, total, halton, st);
    else if (kind == GMT_COST_DUBINS) sample_g<4, 3>(Q, off, nq, total, halton, st);
    else if (d == 2) sample_g<2, 2>(Q, off, nq, total, halton, st);
    else if (d == 3) sample_g<3, 3>(Q, off, nq, total, halton, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
cudaError_t batch_mask(int kind, int d, const QueryDev* Q, const long long* off, int nq, long long tiles,
                       cudaStream_t st) {
    if (tiles == 0) return cudaSuccess;  // every query of the group uses the cell list
    if (kind == GMT_COST_DI) mask_g<GMT_COST_DI, 6>(Q, off, nq, tiles, st);
    else if (kind == GMT_COST_DUBINS) mask_g<GMT_COST_DUBINS, 4>(Q, off, nq, tiles, st);
    else if (d == 2) mask_g<GMT_COST_EUCLID, 2>(Q, off, nq, tiles, st);
    else if (d == 3) mask_g<GMT_COST_EUCLID, 3>(Q, off, nq, tiles, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
// Cell-list stages before the row scan: cell counts, per-query cell scan,
// scatter, row counts (queries without use_cells return at once).  off:
// cumulative node counts; off_cells: cumulative cell counts (cells: their total).
cudaError_t batch_cells_front(int d, const QueryDev* Q, const long long* off, const long long* off_cells, int nq,
                              long long nodes, long long cells, cudaStream_t st) {
    const unsigned tb = (unsigned)((nodes + 255) / 256);
    if (d == 2) batch_cells_count_kernel<2><<<tb, 256, 0, st>>>(Q, off, nq);
    else if (d == 3) batch_cells_count_kernel<3><<<tb, 256, 0, st>>>(Q, off, nq);
    else return cudaErrorInvalidValue;
    batch_cells_scan_kernel<<<nq, 1024, 0, st>>>(Q);
    batch_cells_scatter_kernel<<<tb, 256, 0, st>>>(Q, off, nq);
    if (cells > 0) {
        const size_t smem = cell_tile_smem(d, 0);
        if (d == 2) batch_cells_tile_kernel<2, false><<<(unsigned)cells, kCellWarps * 32, smem, st>>>(Q, off_cells, nq, 0);
        else batch_cells_tile_kernel<3, false><<<(unsigned)cells, kCellWarps * 32, smem, st>>>(Q, off_cells, nq, 0);
    }
    return cudaGetLastError();
}
// words: the largest cell_fill_words of the group's cell-list queries
cudaError_t batch_cells_fill(int d, const QueryDev* Q, const long long* off_cells, int nq, long long cells, int words,
                             cudaStream_t st) {
    if (cells <= 0) return cudaSuccess;
    const size_t smem = cell_tile_smem(d, words);
    if (d == 2) batch_cells_tile_kernel<2, true><<<(unsigned)cells, kCellWarps * 32, smem, st>>>(Q, off_cells, nq, words);
    else if (d == 3) batch_cells_tile_kernel<3, true><<<(unsigned)cells, kCellWarps * 32, smem, st>>>(Q, off_cells, nq, words);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
cudaError_t batch_tile_prefix(const QueryDev* Q, const long long* off_nodes, int nq, long long nodes,
                              cudaStream_t st) {
    batch_tile_prefix_kernel<<<(unsigned)((nodes + 255) / 256), 256, 0, st>>>(Q, off_nodes, nq);
    return cudaGetLastError();
}
cudaError_t batch_fill_tiles(int d, const QueryDev* Q, const long long* off_tiles, int nq, long long tiles,
                             cudaStream_t st) {
    if (tiles <= 0) return cudaSuccess;
    if (d == 2) batch_fill_tile_kernel<2><<<(unsigned)tiles, kMaskRows, 0, st>>>(Q, off_tiles, nq);
    else if (d == 3) batch_fill_tile_kernel<3><<<(unsigned)tiles, kMaskRows, 0, st>>>(Q, off_tiles, nq);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
cudaError_t batch_fill(int kind, int d, const QueryDev* Q, const long long* off, int nq, long long rows,
                       cudaStream_t st) {
    if (kind == GMT_COST_DI) fill_g<GMT_COST_DI, 6>(Q, off, nq, rows, st);
    else if (kind == GMT_COST_DUBINS) fill_g<GMT_COST_DUBINS, 4>(Q, off, nq, rows, st);
    else if (d == 2) fill_g<GMT_COST_EUCLID, 2>(Q, off, nq, rows, st);
    else if (d == 3) fill_g<GMT_COST_EUCLID, 3>(Q, off, nq, rows, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace gmtk

// =========================================================================== host
using namespace gmtk;

namespace {

gmt_status bfail(gmt_status s, const std::string& m) {
    record_error(m.c_str());
    return s;
}
gmt_status bcuda(cudaError_t e, const char* what) {
    return bfail(e == cudaErrorMemoryAllocation ? GMT_ERR_OOM : GMT_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}
#define BCUDA(call, what)                                \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return bcuda(e_, what);   \
    } while (0)

// Device buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t need(size_t bytes) {
        if (p && cap >= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 1);
        if (e == cudaSuccess) cap = bytes ? bytes : 1;
        return e;
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    template <class T> T* as() const { return (T*)p; }
};

float euclid_threshold_b(float r) {
    float t = r * r;
    while (t > 0.0f && std::sqrt(t) >= r) t = std::nextafter(t, 0.0f);
    while (std::sqrt(t) < r) t = std::nextafter(t, INFINITY);
    return t;
}

constexpr size_t kCtlSlotB = 256;
static_assert(sizeof(PlanCtl) <= kCtlSlotB, "control block must fit its slot");

struct Group {
    int kind = 0, d = 0, dp = 0;
    std::vector<int> members;          // query indices
    long long nodes = 0, tiles = 0, tasks = 0, cells = 0;
    int max_n = 0, max_boxes = 0;
    DevBuf desc, off_nodes, off_tiles, off_tasks, off_rows, off_cells, order, args;
    std::vector<int> order_h;
    // lockstep scheme: members [chunk_start[c], chunk_start[c] + chunk_count[c])
    // run in one launch; their node offsets start at lock_base + chunk_base[c]
    std::vector<int> chunk_start, chunk_count, chunk_nodes, chunk_base, chunk_ctl;
    DevBuf lock_base;
    bool any_cells = false;  // some member builds its neighbours with the cell list
    bool any_tiles = false;  // some member fills its CSR by mask tiles
    int cell_words = 0;      // largest fill buffer (words per warp) of those members
    bool any_halton = false; // some member samples with the Halton sequence
};

}  // namespace

struct gmt_batch {
    int q = 0;
    std::vector<gmt_query> queries;
    std::vector<int> N, pitch;
    std::vector<long long> node_base;  // offsets into the caller's parent/cost arrays
    std::vector<long long> E;
    std::vector<QueryDev> qd;
    std::vector<float> r;
    std::vector<Group> groups;
    // arena
    DevBuf X, goal, flags, mask, maskT, counts, rows, edges_i, edges_f, path, ctl, next, slot, tcnt;
    DevBuf cells, cell_info;
    DevBuf s_ocost, s_stamp, s_lists;
    DevBuf l_open, l_glist, l_ocost, l_stamp, l_ctl;
    DevBuf p_args, p_order, p_ecum, p_q, p_ctl, p_scratch;  // pool scheme
    int lock_chunks = 0;
    int max_n = 0;  // largest N of the batch (team scratch slices)
    cudaEvent_t ev_plan[2] = {nullptr, nullptr};  // around the plan stage of every call
    PlanCtl* h_ctl = nullptr;
    int* h_rows = nullptr;  // [q] edge counts, then [q] sampling flags
    size_t h_cap = 0;
    // scheme and launch shape of the plan stage
    int mode = GMT_BATCH_AUTO;
    int cluster = 0, threads = 0;      // 0 = automatic / tuned
    int tuned_mode = GMT_BATCH_AUTO, tuned_cluster = 0, tuned_threads = 0;
    // captured replay
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t* cap_parent = nullptr;
    float* cap_cost = nullptr;
    bool prepared = false;
    int calls_same = 0;
    cudaStream_t cap_stream = nullptr;

    ~gmt_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (h_ctl) cudaFreeHost(h_ctl);
        if (h_rows) cudaFreeHost(h_rows);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (cudaEvent_t e : ev_plan)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

gmt_status check_query(const gmt_query& Qh, int k) {
    const gmt_space& sp = Qh.space;
    const std::string at = " (query " + std::to_string(k) + ")";
    if (sp.kind == GMT_COST_EUCLID) {
        if (!(sp.dim == 2 || sp.dim == 3) || sp.pos_dim != sp.dim)
            return bfail(GMT_ERR_INVALID, "batched geometric queries need dim 2 or 3 and pos_dim == dim" + at);
    } else if (sp.kind == GMT_COST_DI) {
        if (sp.dim != 6 || sp.pos_dim != 3) return bfail(GMT_ERR_INVALID, "double integrator needs dim 6, pos_dim 3" + at);
    } else if (sp.kind == GMT_COST_DUBINS) {
        if (sp.dim != 4 || sp.pos_dim != 3) return bfail(GMT_ERR_INVALID, "Dubins airplane needs dim 4, pos_dim 3" + at);
        if (!(Qh.params.turn_radius > 0.0f) || !std::isfinite(Qh.params.turn_radius) || !(Qh.params.r > 0.0f))
            return bfail(GMT_ERR_INVALID, "a Dubins airplane query needs turn_radius > 0 and r > 0" + at);
    } else {
        return bfail(GMT_ERR_INVALID, "unknown cost kind" + at);
    }
    for (int a = 0; a < sp.dim; ++a)
        if (!(sp.lo[a] < sp.hi[a])) return bfail(GMT_ERR_INVALID, "state bounds need lo < hi" + at);
    if (Qh.boxes.count < 0 || (Qh.boxes.count > 0 && (!Qh.boxes.lo || !Qh.boxes.hi)))
        return bfail(GMT_ERR_INVALID, "bad box arrays" + at);
    const gmt_params& p = Qh.params;
    if (p.n < 1 || p.n > (1 << 24)) return bfail(GMT_ERR_INVALID, "n must be in [1, 2^24]" + at);
    if (!(p.lambda >= 0.0f && p.lambda <= 1.0f)) return bfail(GMT_ERR_INVALID, "lambda must be in [0, 1]" + at);
    if (p.sampler != GMT_SAMPLER_PHILOX && p.sampler != GMT_SAMPLER_HALTON)
        return bfail(GMT_ERR_INVALID, "sampler must be GMT_SAMPLER_PHILOX or GMT_SAMPLER_HALTON" + at);
    if (p.r <= 0.0f && (!(p.eta >= 0.0f) || !(p.mu_free > 0.0f)))
        return bfail(GMT_ERR_INVALID, "r <= 0 needs eta >= 0 and mu_free > 0" + at);
    if (!(p.seg_spacing > 0.0f) || p.traj_points < 2)
        return bfail(GMT_ERR_INVALID, "seg_spacing must be > 0 and traj_points >= 2" + at);
    if (!(Qh.goal.radius >= 0.0f)) return bfail(GMT_ERR_INVALID, "goal radius must be >= 0" + at);
    if (Qh.extra_count < 0 || Qh.extra_count > (1 << 24) ||
        (Qh.extra_count > 0 && (!Qh.extra || Qh.extra_pitch < Qh.extra_count)))
        return bfail(GMT_ERR_INVALID, "appended samples need a DEVICE array [dim][extra_pitch], "
                                      "extra_pitch >= extra_count, extra_count in [0, 2^24]" + at);
    return GMT_OK;
}

void info_from_ctl(const PlanCtl& c, gmt_plan_info* info) {
    std::memset(info, 0, sizeof(*info));
    info->status = c.status;
    info->goal_node = c.goal_node;
    info->path_len = c.path_len;
    info->path_cost = INFINITY;
    if (c.status == GMT_OK && c.goal_node >= 0) {
        const unsigned bits = (unsigned)(c.goal_key >> 32);
        std::memcpy(&info->path_cost, &bits, sizeof(float));
    }
    info->iters = c.iters;
    info->final_i = c.final_i;
    info->push_edges = (int64_t)c.push_edges;
    info->pull_edges = (int64_t)c.pull_edges;
    info->checks = (int64_t)c.checks;
    info->failed = (int64_t)c.failed;
    info->tree_size = (int64_t)c.tree_size;
}

// Under stream capture an event record becomes a graph node only with the
// external flag; outside capture it is an ordinary record.
cudaError_t record_plan_event(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(st, &cs);
    if (err != cudaSuccess) return err;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal)
                                               : cudaEventRecord(e, st);
}

// Untuned choice: teams of 4 CTAs x 512 threads (measured fastest on the
// 256-query uneven batch; the autotuner compares every scheme and shape).
int plan_mode(const gmt_batch* b) {
    if (b->mode != GMT_BATCH_AUTO) return b->mode;
    if (b->tuned_mode != GMT_BATCH_AUTO) return b->tuned_mode;
    return GMT_BATCH_TEAMS;
}

// Does the batch hold a double-integrator or Dubins query?
bool pool_all_kinds(const gmt_batch* b) {
    for (const Group& g : b->groups)
        if (g.kind != GMT_COST_EUCLID) return true;
    return false;
}

// Pool launch shape: (threads, co-resident blocks).
void pool_shape(const gmt_batch* b, int* threads, int* blocks) {
    int t = b->threads > 0 ? b->threads : (b->tuned_threads > 0 ? b->tuned_threads : 256);
    if (t > 256) t = 256;
    *threads = t;
    *blocks = plan_pool_max_blocks(t, pool_all_kinds(b));
}

// Lockstep launch shape for a group: (threads, co-resident blocks).
void lock_shape(const gmt_batch* b, const Group& g, int* threads, int* blocks) {
    const int t = b->threads > 0 ? b->threads : (b->tuned_threads > 0 ? b->tuned_threads : 512);
    *threads = t;
    *blocks = plan_lockstep_max_blocks(g.kind, g.dp, t);
}

// Dynamic shared memory of the batched team kernel: the most any query asks
// for (its staged boxes, or the parent copy of its path walk).
size_t batch_smem(const gmt_batch* b) {
    size_t smem = 16;
    for (int k = 0; k < b->q; ++k) {
        const int dp = b->queries[k].space.pos_dim, nb = b->queries[k].boxes.count;
        smem = std::max(smem, plan_smem_bytes(nb <= smem_box_cap(dp) ? nb : 0, dp, b->N[k]));
    }
    return smem;
}

// Plan-stage launch shape of the teams scheme: (cluster, threads, teams).
void plan_shape(const gmt_batch* b, int* cluster, int* threads, int* teams) {
    int c = b->cluster > 0 ? b->cluster : (b->tuned_cluster > 0 ? b->tuned_cluster : 4);
    int t = b->threads > 0 ? b->threads : (b->tuned_threads > 0 ? b->tuned_threads : 512);
    const size_t smem = batch_smem(b);
    const bool all = pool_all_kinds(b);
    int n = plan_batch_max_teams(t, c, smem, b->max_n, true, all);
    while (n <= 0 && c > 1) {
        c /= 2;
        n = plan_batch_max_teams(t, c, smem, b->max_n, true, all);
    }
    *cluster = c;
    *threads = t;
    *teams = n;
}

// Everything after the edge counts are known: fill + plan + result copy.
// Runs on `st`; records nothing that needs the host in between, so it can be
// captured into a CUDA graph together with the first half (see run_device).
gmt_status enqueue_build_front(gmt_batch* b, cudaStream_t st) {
    BCUDA(cudaMemsetAsync(b->flags.p, 0, b->flags.cap, st), "memset");
    BCUDA(cudaMemsetAsync(b->counts.p, 0, b->counts.cap, st), "memset");
    BCUDA(cudaMemsetAsync(b->cells.p, 0, b->cells.cap, st), "memset");
    BCUDA(cudaMemsetAsync(b->cell_info.p, 0, b->cell_info.cap, st), "memset");
    for (Group& g : b->groups) {
        const int nq = (int)g.members.size();
        const QueryDev* Q = g.desc.as<QueryDev>();
        BCUDA(batch_sample(g.kind, g.d, Q, g.off_nodes.as<long long>(), nq, g.nodes, g.any_halton, st),
              "batched sample kernel");
        BCUDA(batch_mask(g.kind, g.d, Q, g.off_tiles.as<long long>(), nq, g.tiles, st), "batched pair filter");
        if (g.any_tiles)
            BCUDA(batch_tile_prefix(Q, g.off_nodes.as<long long>(), nq, g.nodes, st), "batched tile prefixes");
        if (g.any_cells)
            BCUDA(batch_cells_front(g.d, Q, g.off_nodes.as<long long>(), g.off_cells.as<long long>(), nq, g.nodes,
                                    g.cells, st),
                  "batched cells");
        if (g.kind != GMT_COST_EUCLID) {  // directed costs: the in-neighbour bit matrix and rows
            const long long warps = g.tasks;
            batch_transpose_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(Q, g.off_tasks.as<long long>(), nq);
            BCUDA(cudaGetLastError(), "batched transpose");
        }
        batch_scan_kernel<<<nq, 1024, 0, st>>>(Q, 0);
        if (g.kind != GMT_COST_EUCLID) batch_scan_kernel<<<nq, 1024, 0, st>>>(Q, 1);
        BCUDA(cudaGetLastError(), "batched scan");
    }
    return GMT_OK;
}

gmt_status enqueue_build_back(gmt_batch* b, int32_t* parent, float* cost, cudaStream_t st) {
    for (Group& g : b->groups) {
        const int nq = (int)g.members.size();
        const QueryDev* Q = g.desc.as<QueryDev>();
        if (g.kind == GMT_COST_EUCLID) {  // every all-pairs geometric query fills by mask tiles
            if (g.any_tiles)
                BCUDA(batch_fill_tiles(g.d, Q, g.off_tiles.as<long long>(), nq, g.tiles, st), "batched tiled fill");
        } else {
            BCUDA(batch_fill(g.kind, g.d, Q, g.off_rows.as<long long>(), nq, g.nodes, st), "batched fill");
        }
        if (g.any_cells)
            BCUDA(batch_cells_fill(g.d, Q, g.off_cells.as<long long>(), nq, g.cells, g.cell_words, st),
                  "batched cells");
    }
    // sampling flags of this call (appended samples are read on replays too)
    BCUDA(cudaMemcpyAsync(b->h_rows + b->q, b->flags.p, (size_t)b->q * 4, cudaMemcpyDeviceToHost, st),
          "flag readback");
    BCUDA(cudaMemsetAsync(b->ctl.p, 0, b->ctl.cap, st), "memset");
    for (cudaEvent_t& e : b->ev_plan)
        if (!e) BCUDA(cudaEventCreate(&e), "event");
    BCUDA(record_plan_event(b->ev_plan[0], st), "event");
    if (plan_mode(b) == GMT_BATCH_POOL) {
        int threads, blocks;
        pool_shape(b, &threads, &blocks);
        if (blocks <= 0) return bfail(GMT_ERR_CUDA, "pool plan kernel cannot be resident");
        BCUDA(cudaMemsetAsync(b->p_ctl.p, 0, sizeof(PoolCtl), st), "memset");
        BCUDA(launch_plan_pool(b->p_args.as<PlanArgs>(), b->p_order.as<int>(), b->p_ecum.as<long long>(), b->q,
                               b->p_q.as<PoolQ>(), b->p_ctl.as<PoolCtl>(), pool_all_kinds(b), blocks, threads, st),
              "pool plan kernel");
        BCUDA(record_plan_event(b->ev_plan[1], st), "event");
        BCUDA(cudaMemcpyAsync(b->h_ctl, b->ctl.p, (size_t)b->q * kCtlSlotB, cudaMemcpyDeviceToHost, st),
              "result copy");
        return GMT_OK;
    }
    if (plan_mode(b) == GMT_BATCH_LOCKSTEP) {
        BCUDA(cudaMemsetAsync(b->l_ctl.p, 0, b->l_ctl.cap, st), "memset");
        for (Group& g : b->groups) {
            int threads, blocks;
            lock_shape(b, g, &threads, &blocks);
            if (blocks <= 0) return bfail(GMT_ERR_CUDA, "lockstep plan kernel cannot be resident");
            for (size_t c = 0; c < g.chunk_start.size(); ++c) {
                LockScratch sc;
                sc.ctl = b->l_ctl.as<LockCtl>() + g.chunk_ctl[c];
                sc.open[0] = b->l_open.as<int4>();
                sc.open[1] = sc.open[0] + g.chunk_nodes[c];
                sc.glist[0] = b->l_glist.as<int2>();
                sc.glist[1] = sc.glist[0] + g.chunk_nodes[c];
                sc.ocost = b->l_ocost.as<float>();
                sc.stamp = b->l_stamp.as<int>();
                sc.base = g.lock_base.as<int>() + g.chunk_base[c];
                sc.nodes = g.chunk_nodes[c];
                BCUDA(launch_plan_lockstep(g.kind, g.dp, g.args.as<PlanArgs>() + g.chunk_start[c], g.chunk_count[c], sc,
                                           blocks, threads, st),
                      "lockstep plan kernel");
            }
        }
        BCUDA(record_plan_event(b->ev_plan[1], st), "event");
        BCUDA(cudaMemcpyAsync(b->h_ctl, b->ctl.p, (size_t)b->q * kCtlSlotB, cudaMemcpyDeviceToHost, st),
              "result copy");
        return GMT_OK;
    }
    BCUDA(cudaMemsetAsync(b->next.p, 0, b->next.cap, st), "memset");
    {
        int cluster, threads, teams;
        plan_shape(b, &cluster, &threads, &teams);
        if (teams <= 0) return bfail(GMT_ERR_CUDA, "batched plan kernel cannot be resident");
        if ((size_t)teams > b->slot.cap / 4) return bfail(GMT_ERR_CUDA, "batched plan scratch is too small");
        BatchScratch sc;
        sc.ocost = b->s_ocost.as<float>();
        sc.stamp = b->s_stamp.as<int>();
        sc.lists = b->s_lists.as<int>();
        sc.max_nodes = b->max_n;
        BCUDA(launch_plan_batch(b->p_args.as<PlanArgs>(), b->p_order.as<int>(), b->q, b->next.as<int>(),
                                b->slot.as<int>(), sc, teams, threads, cluster, batch_smem(b), b->max_n,
                                pool_all_kinds(b), st),
              "batched plan kernel");
    }
    BCUDA(record_plan_event(b->ev_plan[1], st), "event");
    (void)parent;
    (void)cost;
    BCUDA(cudaMemcpyAsync(b->h_ctl, b->ctl.p, (size_t)b->q * kCtlSlotB, cudaMemcpyDeviceToHost, st), "result copy");
    return GMT_OK;
}

// Lays out the arena for the queries, runs the front half, reads the edge
// counts, sizes the edge slices, fills the descriptors and plan arguments.
// force_pairs[k] != 0: query k uses the all-pairs test even where the cell list
// would apply (set after a row outgrew the cell list's sort buffer).
gmt_status prepare(gmt_batch* b, int q, const gmt_query* queries, int32_t* parent, float* cost, cudaStream_t st,
                   const std::vector<char>& force_pairs = {}) {
    b->prepared = false;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->q = q;
    b->queries.assign(queries, queries + q);
    b->N.resize(q); b->pitch.resize(q); b->node_base.resize(q + 1); b->E.assign(q, 0); b->qd.resize(q); b->r.resize(q);
    b->groups.clear();
    // groups
    for (int k = 0; k < q; ++k) {
        const gmt_space& sp = queries[k].space;
        Group* g = nullptr;
        for (Group& x : b->groups)
            if (x.kind == sp.kind && x.d == sp.dim) g = &x;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->kind = sp.kind; g->d = sp.dim; g->dp = sp.pos_dim;
        }
        g->members.push_back(k);
    }
    // sizes and offsets
    size_t xs = 0, gs = 0, ms = 0, mts = 0, cs = 0, rs = 0, ps = 0, cls = 0, ts = 0;
    std::vector<size_t> xo(q), go(q), mo(q), mto(q), co(q), ro(q), po(q), clo(q), to(q);
    std::vector<char> use_tiles(q, 0);
    std::vector<CellGrid> cgs(q);
    std::vector<char> use_cells(q, 0);
    b->node_base[0] = 0;
    for (int k = 0; k < q; ++k) {
        const gmt_query& Qh = queries[k];
        const int N = Qh.params.n + 1 + Qh.extra_count;
        const int P = (N + 31) / 32 * 32, W = (N + 31) / 32;
        b->N[k] = N; b->pitch[k] = P;
        b->node_base[k + 1] = b->node_base[k] + N;
        b->r[k] = Qh.params.r > 0.0f ? Qh.params.r
                  : Qh.params.sampler == GMT_SAMPLER_HALTON
                      ? (float)gmt_connection_radius_halton(Qh.params.n, Qh.space.dim, Qh.params.eta, Qh.params.mu_free)
                      : (float)gmt_connection_radius(Qh.params.n, Qh.space.dim, Qh.params.eta, Qh.params.mu_free);
        bool pays = false;
        const unsigned dbg = Qh.params.debug_flags;
        const bool applies = make_cell_grid(Qh.space.kind, Qh.space.dim, Qh.space.lo, Qh.space.hi, b->r[k], N,
                                            true, &cgs[k], &pays);
        if (dbg & GMT_DEBUG_CELLS_LIST) cgs[k].list_only = 1;
        use_cells[k] = applies && !(dbg & GMT_DEBUG_PAIRS_ALL) && (pays || (dbg & GMT_DEBUG_PAIRS_CELLS)) &&
                       !(k < (int)force_pairs.size() && force_pairs[k]);
        xo[k] = xs; xs += (size_t)Qh.space.dim * P;
        go[k] = gs; gs += P;
        if (use_cells[k]) {
            clo[k] = cls;
            cls += 2 * (size_t)N + 2 * (size_t)cgs[k].ncells + 1;
        } else {
            mo[k] = ms; ms += (size_t)W * P;
            if (fill_tiles_apply(Qh.space.kind, Qh.space.dim, N, true)) {
                use_tiles[k] = 1;
                to[k] = ts; ts += (size_t)fill_tiles_per_row(N) * P;
            }
        }
        if (Qh.space.kind != GMT_COST_EUCLID) { mto[k] = mts; mts += (size_t)W * P; }
        co[k] = cs; cs += 2 * (size_t)N;
        ro[k] = rs; rs += 2 * (size_t)(N + 1);
        po[k] = ps; ps += N;
    }
    BCUDA(b->X.need(xs * 4), "arena");
    BCUDA(b->goal.need(gs), "arena");
    BCUDA(b->flags.need((size_t)q * 4), "arena");
    BCUDA(b->mask.need(ms * 4 + 4), "arena");
    BCUDA(b->tcnt.need(ts * 4 + 4), "arena");
    BCUDA(b->cells.need(cls * 4 + 4), "arena");
    BCUDA(b->cell_info.need((size_t)q * 2 * 4), "arena");
    BCUDA(b->maskT.need(mts * 4 + 4), "arena");
    BCUDA(b->counts.need(cs * 4), "arena");
    BCUDA(b->rows.need(rs * 4), "arena");
    BCUDA(b->path.need(ps * 4), "arena");
    BCUDA(b->ctl.need((size_t)q * kCtlSlotB), "arena");
    BCUDA(b->next.need(b->groups.size() * 4), "arena");
    if (b->h_cap < (size_t)q) {
        if (b->h_ctl) cudaFreeHost(b->h_ctl);
        if (b->h_rows) cudaFreeHost(b->h_rows);
        b->h_ctl = nullptr; b->h_rows = nullptr; b->h_cap = 0;
        BCUDA(cudaMallocHost((void**)&b->h_ctl, (size_t)q * kCtlSlotB), "pinned");
        BCUDA(cudaMallocHost((void**)&b->h_rows, (size_t)q * 2 * sizeof(int)), "pinned");
        b->h_cap = q;
    }
    for (int k = 0; k < q; ++k) {
        const gmt_query& Qh = queries[k];
        QueryDev& d = b->qd[k];
        std::memset(&d, 0, sizeof(d));
        SpaceArgs& s = d.s;
        s.kind = Qh.space.kind; s.d = Qh.space.dim; s.dp = Qh.space.pos_dim; s.N = b->N[k]; s.pitch = b->pitch[k];
        s.n_sampled = Qh.params.n + 1;
        for (int a = 0; a < s.d; ++a) {
            s.lo[a] = Qh.space.lo[a]; s.hi[a] = Qh.space.hi[a];
            s.x0[a] = Qh.x_init[a]; s.gc[a] = Qh.goal.center[a];
        }
        s.grho = Qh.goal.radius;
        s.gd = Qh.goal.pos_only ? s.dp : s.d;
        s.key0 = (uint32_t)(Qh.params.seed & 0xffffffffu);
        s.key1 = (uint32_t)(Qh.params.seed >> 32);
        s.stream = 0;
        s.max_attempts = Qh.params.max_attempts > 0 ? Qh.params.max_attempts : 65536;
        s.sampler = Qh.params.sampler;
        s.halton_cap = (long long)s.max_attempts + 64LL * s.n_sampled;
        s.r = b->r[k];
        s.r2_threshold = euclid_threshold_b(s.r);
        s.rho = s.kind == GMT_COST_DUBINS ? Qh.params.turn_radius : 0.0f;
        d.boxes = BoxArgs{Qh.boxes.count, Qh.boxes.lo, Qh.boxes.hi};
        d.extra = Qh.extra_count > 0 ? Qh.extra : nullptr;
        d.extra_pitch = Qh.extra_pitch;
        d.X = b->X.as<float>() + xo[k];
        d.is_goal = b->goal.as<uint8_t>() + go[k];
        d.flags = b->flags.as<int>() + k;
        d.mask = use_cells[k] ? nullptr : b->mask.as<uint32_t>() + mo[k];
        d.tile_cnt = use_tiles[k] ? b->tcnt.as<int>() + to[k] : nullptr;
        d.use_cells = use_cells[k];
        d.cg = cgs[k];
        if (use_cells[k]) {
            const size_t N = (size_t)s.N;
            d.cell_of = b->cells.as<int>() + clo[k];
            d.cell_sorted = d.cell_of + N;
            d.cell_cnt = d.cell_sorted + N;
            d.cell_start = d.cell_cnt + cgs[k].ncells;
        }
        d.cell_info = b->cell_info.as<int>() + 2 * k;
        d.maskT = s.kind != GMT_COST_EUCLID ? b->maskT.as<uint32_t>() + mto[k] : nullptr;
        d.out_count = b->counts.as<int>() + co[k];
        d.in_count = d.out_count + s.N;
        d.out_row = b->rows.as<int>() + ro[k];
        d.in_row = s.kind != GMT_COST_EUCLID ? d.out_row + (s.N + 1) : d.out_row;
        d.edge_cap = 0;
    }
    // per-group work offsets and descriptors
    for (Group& g : b->groups) {
        const int nq = (int)g.members.size();
        std::vector<long long> on(nq + 1, 0), ot(nq + 1, 0), ow(nq + 1, 0), oc(nq + 1, 0);
        std::vector<QueryDev> dq(nq);
        g.max_n = 0; g.max_boxes = 0;
        g.any_cells = false;
        g.any_tiles = false;
        g.cell_words = 0;
        g.any_halton = false;
        for (int i = 0; i < nq; ++i) {
            const int k = g.members[i];
            const int N = b->N[k], W = (N + 31) / 32;
            g.any_cells = g.any_cells || use_cells[k];
            g.any_tiles = g.any_tiles || b->qd[k].tile_cnt != nullptr;
            g.any_halton = g.any_halton || queries[k].params.sampler == GMT_SAMPLER_HALTON;
            if (use_cells[k]) g.cell_words = std::max(g.cell_words, cell_fill_words(cgs[k], N));
            const long long tiles =
                use_cells[k] ? 0
                : g.kind == GMT_COST_DI
                    ? (long long)((N + kDIRows - 1) / kDIRows) * ((W + kDIWords - 1) / kDIWords)
                : g.kind == GMT_COST_DUBINS
                    ? (long long)((N + kDubRows - 1) / kDubRows) * ((W + kDubWords - 1) / kDubWords)
                    : (long long)((N + kMaskRows - 1) / kMaskRows) * ((W + kMaskWords - 1) / kMaskWords);
            on[i + 1] = on[i] + N;
            oc[i + 1] = oc[i] + (use_cells[k] ? cgs[k].ncells : 0);
            ot[i + 1] = ot[i] + tiles;
            ow[i + 1] = ow[i] + (long long)W * W;
            g.max_n = std::max(g.max_n, N);
            g.max_boxes = std::max(g.max_boxes, queries[k].boxes.count);
            dq[i] = b->qd[k];
        }
        g.nodes = on[nq]; g.tiles = ot[nq]; g.tasks = ow[nq]; g.cells = oc[nq];
        BCUDA(g.desc.need(nq * sizeof(QueryDev)), "descriptors");
        BCUDA(g.off_nodes.need((nq + 1) * 8), "descriptors");
        BCUDA(g.off_tiles.need((nq + 1) * 8), "descriptors");
        BCUDA(g.off_tasks.need((nq + 1) * 8), "descriptors");
        BCUDA(g.off_rows.need((nq + 1) * 8), "descriptors");
        BCUDA(g.off_cells.need((nq + 1) * 8), "descriptors");
        BCUDA(cudaMemcpyAsync(g.desc.p, dq.data(), nq * sizeof(QueryDev), cudaMemcpyHostToDevice, st), "upload");
        BCUDA(cudaMemcpyAsync(g.off_nodes.p, on.data(), (nq + 1) * 8, cudaMemcpyHostToDevice, st), "upload");
        BCUDA(cudaMemcpyAsync(g.off_tiles.p, ot.data(), (nq + 1) * 8, cudaMemcpyHostToDevice, st), "upload");
        BCUDA(cudaMemcpyAsync(g.off_tasks.p, ow.data(), (nq + 1) * 8, cudaMemcpyHostToDevice, st), "upload");
        BCUDA(cudaMemcpyAsync(g.off_rows.p, on.data(), (nq + 1) * 8, cudaMemcpyHostToDevice, st), "upload");
        BCUDA(cudaMemcpyAsync(g.off_cells.p, oc.data(), (nq + 1) * 8, cudaMemcpyHostToDevice, st), "upload");
        BCUDA(cudaStreamSynchronize(st), "upload");  // host vectors go out of scope
    }
    gmt_status s = enqueue_build_front(b, st);
    if (s != GMT_OK) return s;
    // edge counts: out_row[N] (and in_row[N]) of every query
    for (int k = 0; k < q; ++k)
        BCUDA(cudaMemcpyAsync(b->h_rows + k, b->qd[k].out_row + b->N[k], sizeof(int), cudaMemcpyDeviceToHost, st),
              "edge count readback");
    std::vector<int> flags(q), cell_info(2 * (size_t)q);
    BCUDA(cudaMemcpyAsync(flags.data(), b->flags.p, (size_t)q * 4, cudaMemcpyDeviceToHost, st), "flag readback");
    BCUDA(cudaMemcpyAsync(cell_info.data(), b->cell_info.p, (size_t)q * 8, cudaMemcpyDeviceToHost, st),
          "cell readback");
    BCUDA(cudaStreamSynchronize(st), "batched graph build");
    {
        // a row too long for the cell list's sort buffer: that query takes the
        // all-pairs test instead, and the batch is prepared again
        std::vector<char> force(force_pairs);
        force.resize(q, 0);
        bool again = false;
        for (int k = 0; k < q; ++k)
            if (use_cells[k] && !cell_fill_fits(cgs[k], b->N[k], cell_info[2 * k])) {
                force[k] = 1;
                again = true;
            }
        if (again) return prepare(b, q, queries, parent, cost, st, force);
    }
    for (int k = 0; k < q; ++k) {
        if (flags[k] & kSampleBadInit)
            return bfail(GMT_ERR_INVALID, "x_init outside X or in an obstacle (query " + std::to_string(k) + ")");
        if (flags[k] & kSampleExhausted)
            return bfail(GMT_ERR_INVALID, "sampling exhausted max_attempts (query " + std::to_string(k) + ")");
        if (flags[k] & kSampleBadAppend)
            return bfail(GMT_ERR_INVALID,
                         "an appended sample is outside X or in X_obs (query " + std::to_string(k) + ")");
    }
    // edge slices: ints (columns) and floats; a Dubins query's float slice
    // starts with its in-edge words (4 floats each), kept 16-byte aligned
    size_t ei = 0, ef = 0;
    std::vector<size_t> eo(q), fo(q);
    for (int k = 0; k < q; ++k) {
        b->E[k] = b->h_rows[k];
        const size_t E = (size_t)b->E[k];
        const int kind = queries[k].space.kind;
        eo[k] = ei;
        ei += E * (kind == GMT_COST_EUCLID ? 1 : 2);
        fo[k] = ef;
        ef += (kind == GMT_COST_EUCLID ? E : kind == GMT_COST_DI ? 4 * E : 6 * E);
        ef = (ef + 3) / 4 * 4;
    }
    BCUDA(b->edges_i.need(ei * 4 + 4), "edge arena");
    BCUDA(b->edges_f.need(ef * 4 + 16), "edge arena");
    for (int k = 0; k < q; ++k) {
        QueryDev& d = b->qd[k];
        const size_t E = (size_t)b->E[k];
        const bool di = d.s.kind == GMT_COST_DI, dub = d.s.kind == GMT_COST_DUBINS, directed = di || dub;
        float* f = b->edges_f.as<float>() + fo[k];
        d.in_path = dub ? f : nullptr;
        if (dub) f += 4 * E;
        d.out_col = b->edges_i.as<int>() + eo[k];
        d.out_cost = f;
        d.out_tau = di ? f + E : nullptr;
        d.in_col = directed ? d.out_col + E : d.out_col;
        d.in_cost = di ? f + 2 * E : dub ? f + E : d.out_cost;
        d.in_tau = di ? f + 3 * E : nullptr;
        d.edge_cap = (long long)E;
    }
    // plan arguments, order (largest edge count first), scratch
    int max_n = 0;
    for (Group& g : b->groups) {
        const int nq = (int)g.members.size();
        std::vector<QueryDev> dq(nq);
        std::vector<PlanArgs> pa(nq);
        for (int i = 0; i < nq; ++i) {
            const int k = g.members[i];
            const QueryDev& d = b->qd[k];
            const gmt_query& Qh = queries[k];
            dq[i] = d;
            PlanArgs& a = pa[i];
            std::memset(&a, 0, sizeof(a));
            a.kind = d.s.kind; a.d = d.s.d; a.dp = d.s.dp; a.N = d.s.N; a.pitch = d.s.pitch;
            a.X = d.X; a.is_goal = d.is_goal;
            a.out_row = d.out_row; a.out_col = d.out_col;
            a.in_row = d.in_row; a.in_col = d.in_col; a.in_cost = d.in_cost; a.in_tau = d.in_tau;
            a.in_path = d.in_path;
            a.rho = d.s.rho;
            a.boxes = d.boxes;
            for (int c = 0; c < 3 && c < d.s.dp; ++c) { a.pos_lo[c] = Qh.space.lo[c]; a.pos_hi[c] = Qh.space.hi[c]; }
            a.r = d.s.r;
            a.delta = Qh.params.lambda * d.s.r;
            a.seg_spacing = Qh.params.seg_spacing;
            a.traj_points = Qh.params.traj_points;
            a.max_iters = Qh.params.max_iters > 0 ? Qh.params.max_iters : d.s.N + 1;
            a.spin_limit = Qh.params.spin_limit;
            a.debug_flags = 0;
            a.cost = cost + b->node_base[k];
            a.parent = parent + b->node_base[k];
            a.path = b->path.as<int>() + po[k];
            a.ctl = (PlanCtl*)(b->ctl.as<unsigned char>() + (size_t)k * kCtlSlotB);
            a.check_edges = 1;
            a.edge_cap = d.edge_cap;
        }
        g.order_h.resize(nq);
        std::iota(g.order_h.begin(), g.order_h.end(), 0);
        std::stable_sort(g.order_h.begin(), g.order_h.end(),
                         [&](int x, int y) { return b->E[g.members[x]] > b->E[g.members[y]]; });
        BCUDA(cudaMemcpyAsync(g.desc.p, dq.data(), nq * sizeof(QueryDev), cudaMemcpyHostToDevice, st), "upload");
        BCUDA(g.args.need(nq * sizeof(PlanArgs)), "plan arguments");
        BCUDA(g.order.need(nq * sizeof(int)), "plan order");
        BCUDA(cudaMemcpyAsync(g.args.p, pa.data(), nq * sizeof(PlanArgs), cudaMemcpyHostToDevice, st), "upload");
        BCUDA(cudaMemcpyAsync(g.order.p, g.order_h.data(), nq * sizeof(int), cudaMemcpyHostToDevice, st), "upload");
        BCUDA(cudaStreamSynchronize(st), "upload");
        max_n = std::max(max_n, g.max_n);
    }
    // pool scheme: every query with its own scratch (two snapshot buffers,
    // stamps, lists), all queries in one launch, largest edge count first
    {
        std::vector<PlanArgs> all(q);
        for (Group& g : b->groups) {
            std::vector<PlanArgs> pa(g.members.size());
            BCUDA(cudaMemcpyAsync(pa.data(), g.args.p, pa.size() * sizeof(PlanArgs), cudaMemcpyDeviceToHost, st),
                  "download");
            BCUDA(cudaStreamSynchronize(st), "download");
            for (size_t i = 0; i < pa.size(); ++i) all[g.members[i]] = pa[i];
        }
        size_t words = 0;
        std::vector<size_t> so(q);
        for (int k = 0; k < q; ++k) {
            so[k] = words;
            const size_t N = (size_t)b->N[k];
            words += (3 * N + plan_list_stride(N) + 3) / 4 * 4;  // 16-byte aligned slices
        }
        BCUDA(b->p_scratch.need(words * 4 + 16), "pool scratch");
        for (int k = 0; k < q; ++k) {
            const size_t N = (size_t)b->N[k];
            int* base = b->p_scratch.as<int>() + so[k];
            PlanArgs& a = all[k];
            a.ocost = (float*)base;
            a.stamp = base + 2 * N;
            assign_plan_lists(a, base + (3 * N + 3) / 4 * 4, N);
        }
        std::vector<int> order(q);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->E[x] > b->E[y]; });
        std::vector<long long> ecum(q + 1, 0);
        for (int i = 0; i < q; ++i) ecum[i + 1] = ecum[i] + std::max<long long>(b->E[order[i]], 1);
        BCUDA(b->p_args.need((size_t)q * sizeof(PlanArgs)), "pool arguments");
        BCUDA(b->p_order.need((size_t)q * sizeof(int)), "pool arguments");
        BCUDA(b->p_ecum.need((size_t)(q + 1) * sizeof(long long)), "pool arguments");
        BCUDA(b->p_q.need((size_t)q * sizeof(PoolQ)), "pool arguments");
        BCUDA(b->p_ctl.need(sizeof(PoolCtl)), "pool arguments");
        BCUDA(cudaMemcpyAsync(b->p_args.p, all.data(), (size_t)q * sizeof(PlanArgs), cudaMemcpyHostToDevice, st),
              "upload");
        BCUDA(cudaMemcpyAsync(b->p_order.p, order.data(), (size_t)q * sizeof(int), cudaMemcpyHostToDevice, st),
              "upload");
        BCUDA(cudaMemcpyAsync(b->p_ecum.p, ecum.data(), (size_t)(q + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                              st),
              "upload");
        BCUDA(cudaStreamSynchronize(st), "upload");
    }
    // lockstep chunks: up to kLockMaxQueries members per launch
    size_t lock_nodes = 1;
    int chunks = 0;
    for (Group& g : b->groups) {
        const int nq = (int)g.members.size();
        g.chunk_start.clear(); g.chunk_count.clear(); g.chunk_nodes.clear(); g.chunk_base.clear(); g.chunk_ctl.clear();
        std::vector<int> base;
        for (int c0 = 0; c0 < nq; c0 += kLockMaxQueries) {
            const int cnt = std::min(kLockMaxQueries, nq - c0);
            g.chunk_start.push_back(c0);
            g.chunk_count.push_back(cnt);
            g.chunk_base.push_back((int)base.size());
            g.chunk_ctl.push_back(chunks++);
            long long acc = 0;
            for (int i = 0; i < cnt; ++i) {
                base.push_back((int)acc);
                acc += b->N[g.members[c0 + i]];
            }
            if (acc > (1ll << 30)) return bfail(GMT_ERR_INVALID, "too many nodes in one lockstep launch");
            base.push_back((int)acc);
            g.chunk_nodes.push_back((int)acc);
            lock_nodes = std::max(lock_nodes, (size_t)acc);
        }
        BCUDA(g.lock_base.need(base.size() * 4), "lockstep offsets");
        BCUDA(cudaMemcpyAsync(g.lock_base.p, base.data(), base.size() * 4, cudaMemcpyHostToDevice, st), "upload");
        BCUDA(cudaStreamSynchronize(st), "upload");
    }
    BCUDA(b->l_open.need(2 * lock_nodes * sizeof(int4)), "lockstep scratch");
    BCUDA(b->l_glist.need(2 * lock_nodes * sizeof(int2)), "lockstep scratch");
    BCUDA(b->l_ocost.need(lock_nodes * 4), "lockstep scratch");
    BCUDA(b->l_stamp.need(lock_nodes * 4), "lockstep scratch");
    BCUDA(b->l_ctl.need((size_t)chunks * sizeof(LockCtl)), "lockstep scratch");
    b->lock_chunks = chunks;
    // scratch for the most teams any shape can run
    int max_teams = 0;
    b->max_n = max_n;
    {
        const size_t smem = batch_smem(b);
        const bool all = pool_all_kinds(b);
        for (int c : {1, 2, 4, 8, 16})
            for (int t : {256, 512, 1024})
                max_teams = std::max(max_teams, plan_batch_max_teams(t, c, smem, max_n, false, all));
    }
    cudaGetLastError();
    if (max_teams <= 0) return bfail(GMT_ERR_CUDA, "batched plan kernel cannot be resident");
    BCUDA(b->s_ocost.need((size_t)max_teams * 2 * max_n * 4), "scratch");
    BCUDA(b->s_stamp.need((size_t)max_teams * max_n * 4), "scratch");
    BCUDA(b->s_lists.need((size_t)max_teams * plan_list_stride(max_n) * 4), "scratch");
    BCUDA(b->slot.need((size_t)max_teams * 4), "scratch");
    // scratch slices are indexed by team id, so every group may use all of it
    for (Group& g : b->groups) g.max_n = max_n;
    b->prepared = true;
    b->cap_parent = parent;
    b->cap_cost = cost;
    return GMT_OK;
}

bool same_request(const gmt_batch* b, int q, const gmt_query* queries, int32_t* parent, float* cost) {
    return b->prepared && b->q == q && b->cap_parent == parent && b->cap_cost == cost &&
           std::memcmp(b->queries.data(), queries, (size_t)q * sizeof(gmt_query)) == 0;
}

gmt_status finish(gmt_batch* b, gmt_plan_info* infos, cudaStream_t st) {
    BCUDA(cudaStreamSynchronize(st), "batched plan");
    gmt_status worst = GMT_OK;
    for (int k = 0; k < b->q; ++k) {
        const PlanCtl& c = *(const PlanCtl*)((const unsigned char*)b->h_ctl + (size_t)k * kCtlSlotB);
        info_from_ctl(c, &infos[k]);
        if (b->h_rows[b->q + k] & kSampleBadAppend) infos[k].status = GMT_ERR_INVALID;
        if (infos[k].status < 0 && worst == GMT_OK) worst = (gmt_status)infos[k].status;
    }
    if (worst != GMT_OK) return bfail(worst, "at least one query failed (see its info.status)");
    return GMT_OK;
}

}  // namespace

extern "C" {

gmt_status gmt_plan_batch(int32_t q, const gmt_query* queries, gmt_batch** batch, int32_t* parent, float* cost,
                          gmt_plan_info* infos, gmt_stream stream) {
    if (q < 1 || !queries || !batch || !parent || !cost || !infos)
        return bfail(GMT_ERR_INVALID, "q >= 1 and non-NULL queries, batch, parent, cost and infos are required");
    for (int k = 0; k < q; ++k) {
        gmt_status s = check_query(queries[k], k);
        if (s != GMT_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool fresh = *batch == nullptr;
    gmt_batch* b = fresh ? new gmt_batch() : *batch;
    if (fresh) *batch = b;
    if (same_request(b, q, queries, parent, cost)) {
        // replay: capture the device sequence once, then launch the graph
        if (!b->exec) {
            if (!b->cap_stream) BCUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream");
            BCUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture");
            gmt_status s = enqueue_build_front(b, b->cap_stream);
            if (s == GMT_OK) s = enqueue_build_back(b, parent, cost, b->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
            if (s != GMT_OK) { if (g) cudaGraphDestroy(g); return s; }
            if (e != cudaSuccess) return bcuda(e, "graph capture");
            b->graph = g;
            BCUDA(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
        }
        BCUDA(cudaGraphLaunch(b->exec, st), "graph launch");
        return finish(b, infos, st);
    }
    gmt_status s = prepare(b, q, queries, parent, cost, st);
    if (s != GMT_OK) return s;
    s = enqueue_build_back(b, parent, cost, st);
    if (s != GMT_OK) return s;
    return finish(b, infos, st);
}

gmt_status gmt_batch_get_view(const gmt_batch* b, int32_t k, gmt_graph_view* v, int32_t** path) {
    if (!b || !v || !b->prepared || k < 0 || k >= b->q) return bfail(GMT_ERR_INVALID, "no such prepared query");
    const QueryDev& d = b->qd[k];
    std::memset(v, 0, sizeof(*v));
    v->kind = d.s.kind; v->dim = d.s.d; v->pos_dim = d.s.dp; v->N = d.s.N; v->x_pitch = d.s.pitch;
    v->E = b->E[k]; v->r = d.s.r;
    v->X = d.X; v->is_goal = d.is_goal;
    v->out_row = d.out_row; v->out_col = d.out_col; v->out_cost = d.out_cost;
    v->in_row = d.in_row; v->in_col = d.in_col; v->in_cost = d.in_cost;
    v->out_tau = d.out_tau; v->in_tau = d.in_tau;
    v->turn_radius = d.s.rho;
    v->in_path = d.in_path;
    if (path) *path = b->path.as<int>() + (b->node_base[k]);
    return GMT_OK;
}

gmt_status gmt_batch_set_mode(gmt_batch* b, int32_t mode) {
    if (!b) return bfail(GMT_ERR_INVALID, "batch is NULL");
    if (mode != GMT_BATCH_AUTO && mode != GMT_BATCH_TEAMS && mode != GMT_BATCH_LOCKSTEP && mode != GMT_BATCH_POOL)
        return bfail(GMT_ERR_INVALID,
                     "mode must be GMT_BATCH_AUTO, GMT_BATCH_TEAMS, GMT_BATCH_LOCKSTEP or GMT_BATCH_POOL");
    b->mode = mode;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    return GMT_OK;
}

gmt_status gmt_batch_set_launch(gmt_batch* b, int32_t cluster, int32_t threads) {
    if (!b) return bfail(GMT_ERR_INVALID, "batch is NULL");
    if (cluster < 0 || cluster > 16 || (cluster & (cluster - 1)) != 0)
        return bfail(GMT_ERR_INVALID, "cluster must be 0 or a power of two up to 16");
    if (threads != 0 && (threads < 128 || threads > 1024 || threads % 32 != 0))
        return bfail(GMT_ERR_INVALID, "threads must be 0 or a multiple of 32 in [128, 1024]");
    b->cluster = cluster;
    b->threads = threads;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    return GMT_OK;
}

gmt_status gmt_batch_get_launch(const gmt_batch* b, int32_t* mode, int32_t* cluster, int32_t* threads) {
    if (!b) return bfail(GMT_ERR_INVALID, "batch is NULL");
    const int m = plan_mode(b);
    int c = 0, t = 0;
    if (m == GMT_BATCH_POOL) {
        int blocks = 0;
        pool_shape(b, &t, &blocks);
    } else if (m == GMT_BATCH_LOCKSTEP) {
        t = b->threads > 0 ? b->threads : (b->tuned_threads > 0 ? b->tuned_threads : 512);
    } else {
        int teams = 0;
        plan_shape(b, &c, &t, &teams);
    }
    if (mode) *mode = m;
    if (cluster) *cluster = c;
    if (threads) *threads = t;
    return GMT_OK;
}

gmt_status gmt_batch_autotune(gmt_batch* b, gmt_stream stream, int32_t* best_cluster, int32_t* best_threads,
                              float* best_ms) {
    if (!b || !b->prepared) return bfail(GMT_ERR_INVALID, "autotune needs a batch planned once");
    cudaStream_t st = (cudaStream_t)stream;
    const int keep_m = b->mode, keep_c = b->cluster, keep_t = b->threads;
    cudaEvent_t e0, e1;
    BCUDA(cudaEventCreate(&e0), "event");
    BCUDA(cudaEventCreate(&e1), "event");
    float best = INFINITY;
    int bm = GMT_BATCH_AUTO, bc = 0, bt = 0;
    struct Shape { int mode, cluster, threads; };
    std::vector<Shape> shapes;
    for (int t : {128, 256}) shapes.push_back({GMT_BATCH_POOL, 0, t});
    for (int t : {256, 512, 1024}) shapes.push_back({GMT_BATCH_LOCKSTEP, 0, t});
    for (int c : {1, 2, 4, 8, 16})
        for (int t : {256, 512, 1024}) shapes.push_back({GMT_BATCH_TEAMS, c, t});
    gmt_status fail = GMT_OK;
    for (const Shape& sh : shapes) {
        b->mode = sh.mode;
        b->cluster = sh.cluster;
        b->threads = sh.threads;
        bool ok = true;
        if (sh.mode == GMT_BATCH_POOL) {
            int tt, blocks;
            pool_shape(b, &tt, &blocks);
            if (blocks <= 0) ok = false;
        }
        for (Group& g : b->groups) {
            if (sh.mode == GMT_BATCH_POOL) break;
            if (sh.mode == GMT_BATCH_LOCKSTEP) {
                int tt, blocks;
                lock_shape(b, g, &tt, &blocks);
                if (blocks <= 0) ok = false;
            } else {
                int cc, tt, teams;
                plan_shape(b, &cc, &tt, &teams);
                if (cc != sh.cluster || teams <= 0) ok = false;
            }
        }
        cudaGetLastError();
        if (!ok) continue;
        float ms_sum = 0.0f;
        for (int rep = 0; rep < 2 && fail == GMT_OK; ++rep) {
            cudaError_t e = cudaEventRecord(e0, st);
            if (e != cudaSuccess) { fail = bcuda(e, "event"); break; }
            fail = enqueue_build_back(b, b->cap_parent, b->cap_cost, st);
            if (fail != GMT_OK) break;
            e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) { fail = bcuda(e, "event"); break; }
            if (rep > 0) ms_sum += ms;
        }
        if (fail != GMT_OK) break;
        if (ms_sum < best) { best = ms_sum; bm = sh.mode; bc = sh.cluster; bt = sh.threads; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->mode = keep_m;
    b->cluster = keep_c;
    b->threads = keep_t;
    if (fail != GMT_OK) return fail;
    b->tuned_mode = bm;
    b->tuned_cluster = bc;
    b->tuned_threads = bt;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    if (best_cluster) *best_cluster = bc;
    if (best_threads) *best_threads = bt;
    if (best_ms) *best_ms = best;
    return GMT_OK;
}

gmt_status gmt_batch_last_plan_ms(const gmt_batch* b, float* ms) {
    if (!b || !ms || !b->ev_plan[0] || !b->ev_plan[1]) return bfail(GMT_ERR_INVALID, "no plan stage has run");
    BCUDA(cudaEventElapsedTime(ms, b->ev_plan[0], b->ev_plan[1]), "event");
    return GMT_OK;
}

void gmt_batch_free(gmt_batch* b) { delete b; }

}  // extern "C"
