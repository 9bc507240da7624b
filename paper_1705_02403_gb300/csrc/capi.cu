// C ABI of the planner (include/gmt.h): argument checks, device buffers of the
// opaque handles, and the launch sequence of every entry point.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"

using namespace gmtk;

namespace {

thread_local std::string g_last_error;

gmt_status fail(gmt_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

gmt_status cuda_fail(cudaError_t e, const char* what) {
    const gmt_status s = e == cudaErrorMemoryAllocation ? GMT_ERR_OOM : GMT_ERR_CUDA;
    return fail(s, std::string(what) + ": " + cudaGetErrorString(e));
}

#define GMT_CUDA(call, what)                              \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

template <typename T>
cudaError_t grow(T** p, size_t* cap, size_t need) {
    if (*p && *cap >= need) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (need == 0) need = 1;
    cudaError_t e = cudaMalloc((void**)p, need * sizeof(T));
    if (e == cudaSuccess) *cap = need;
    return e;
}

// Pinned host memory mapped into the device address space (the device writes
// results there directly; the host reads them after synchronising).
template <class T>
cudaError_t alloc_mapped(T** host, T** dev, size_t n) {
    cudaError_t e = cudaHostAlloc((void**)host, n * sizeof(T), cudaHostAllocMapped);
    if (e != cudaSuccess) {
        *host = nullptr;
        return e;
    }
    std::memset(*host, 0, n * sizeof(T));
    e = cudaHostGetDevicePointer((void**)dev, *host, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(*host);
        *host = nullptr;
    }
    return e;
}

// Smallest float t with sqrtf(t) >= r: for s >= 0, sqrtf(s) < r  <=>  s < t,
// because correctly rounded square root is monotone.
float euclid_threshold(float r) {
    float t = r * r;
    while (t > 0.0f && std::sqrt(t) >= r) t = std::nextafter(t, 0.0f);
    while (std::sqrt(t) < r) t = std::nextafter(t, INFINITY);
    return t;
}

}  // namespace

namespace gmtk {
void record_error(const char* msg) { g_last_error = msg; }
}  // namespace gmtk

// Device ints at the front of a graph's count block (see gmt_graph::flags).
constexpr int kFlagInts = 8;

struct gmt_graph {
    int kind = 0, d = 0, dp = 0, N = 0, pitch = 0;
    long long E = 0;
    float r = 0.0f;
    float rho = 0.0f;   // Dubins airplane turning radius the costs were built with
    float pos_lo[3] = {0, 0, 0}, pos_hi[3] = {0, 0, 0};
    int plan_blocks = 0, plan_threads = 0, plan_cluster = 0;   // 0 = automatic
    int auto_cluster = -1;                                     // probed once
    float* X = nullptr;            size_t cap_X = 0;
    uint8_t* is_goal = nullptr;    size_t cap_is_goal = 0;
    int* out_row = nullptr;        size_t cap_out_row = 0;
    int* in_row_own = nullptr;     size_t cap_in_row_own = 0;
    // one block, zeroed by one memset per build: [flags: kFlagInts][out_count: N][in_count: N]
    int* counts = nullptr;         size_t cap_counts = 0;
    int* out_count = nullptr;      // views into `counts`
    int* in_count = nullptr;
    int* out_col = nullptr;        size_t cap_out_col = 0;
    float* out_cost = nullptr;     size_t cap_out_cost = 0;
    int* in_col_own = nullptr;     size_t cap_in_col_own = 0;
    float* in_cost_own = nullptr;  size_t cap_in_cost_own = 0;
    float* out_tau = nullptr;      size_t cap_out_tau = 0;
    float* in_tau = nullptr;       size_t cap_in_tau = 0;
    float* in_path = nullptr;      size_t cap_in_path = 0;   // Dubins airplane: [E][4] (t, p, q, word bits)
    uint32_t* mask = nullptr;      size_t cap_mask = 0;
    uint32_t* maskT = nullptr;     size_t cap_maskT = 0;
    int* tile_cnt = nullptr;       size_t cap_tile_cnt = 0;  // per-tile row counts of the tiled fill
    // directed costs: the pair filter's edge list (row, column, cost, arrival
    // time), the Dubins words at the same slots, and the word prefixes of mask
    // and maskT that place them
    int4* elist = nullptr;         size_t cap_elist = 0;
    float4* epath = nullptr;       size_t cap_epath = 0;
    int* wpre = nullptr;           size_t cap_wpre = 0;
    int* wpreT = nullptr;          size_t cap_wpreT = 0;
    // [sample flags, max row length, -, fill ticket, cell row overflow, edge list count, -, -]
    int* flags = nullptr;
    // cell-list neighbour build
    int* cell_of = nullptr;        size_t cap_cell_of = 0;
    int* cell_sorted = nullptr;    size_t cap_cell_sorted = 0;
    int* cell_cnt = nullptr;       size_t cap_cell_cnt = 0;
    int* cell_start = nullptr;     size_t cap_cell_start = 0;
    bool used_cells = false;
    // box grid of the last plan (many boxes)
    int* grid_cnt = nullptr;       size_t cap_grid_cnt = 0;
    int* grid_start = nullptr;     size_t cap_grid_start = 0;
    int* grid_list = nullptr;      size_t cap_grid_list = 0;
    int* grid_big = nullptr;       size_t cap_grid_big = 0;
    int* halton = nullptr;         size_t cap_halton = 0;    // multi-block Halton sampler scratch (ints)
    // plan workspace
    float* ocost = nullptr;        size_t cap_ocost = 0;
    int* stamp = nullptr;          size_t cap_stamp = 0;
    int* lists = nullptr;          size_t cap_lists = 0;
    PlanCtl* ctl = nullptr;        size_t cap_ctl = 0;
    // pinned host mirrors
    PlanCtl* h_ctl = nullptr;      // mapped into the device: d_ctl, d_scalars
    int* h_scalars = nullptr;
    PlanCtl* d_ctl = nullptr;
    int* d_scalars = nullptr;
    // An asynchronous build (gmt_build_graph_async) not yet confirmed: its fill
    // wrote into the edge arrays of earlier builds (`pending_cap` edges); the
    // flags and edge count are read by the next plan or view, which rebuilds
    // synchronously from the kept inputs if the edges did not fit.
    bool pending = false;
    long long pending_cap = 0;
    cudaStream_t pending_stream = nullptr;
    gmt_space p_space;
    gmt_boxes p_boxes;
    float p_x_init[GMT_MAX_DIM];
    gmt_goal p_goal;
    gmt_params p_params;
    // profiling: event pairs around each kernel group
    enum { kSample, kPair, kTranspose, kScan, kFill, kPlan, kStages };
    int profiling = 0;  // 0 off, 1 every stage, 2 the plan kernel only
    bool stage_ran[kStages] = {};
    cudaEvent_t ev[kStages][2] = {};
    int last_blocks = 0, last_threads = 0;

    cudaError_t mark(int stage, int which, cudaStream_t st) {
        if (!profiling || (profiling == 2 && stage != kPlan)) return cudaSuccess;
        if (!ev[stage][which]) {
            cudaError_t e = cudaEventCreate(&ev[stage][which]);
            if (e != cudaSuccess) return e;
        }
        if (which == 1) stage_ran[stage] = true;
        return cudaEventRecord(ev[stage][which], st);
    }

    // costs that are not symmetric (double integrator, Dubins airplane) keep
    // their own in-CSR
    bool directed() const { return kind != GMT_COST_EUCLID; }
    const int* in_row() const { return directed() ? in_row_own : out_row; }
    const int* in_col() const { return directed() ? in_col_own : out_col; }
    const float* in_cost() const { return directed() ? in_cost_own : out_cost; }

    ~gmt_graph() {
        void* dev[] = {X, is_goal, out_row, in_row_own, counts, out_col, out_cost, in_col_own,
                       in_cost_own, out_tau, in_tau, in_path, mask, maskT, tile_cnt, elist, epath, wpre, wpreT,
                       cell_of, cell_sorted, cell_cnt,
                       cell_start, grid_cnt, grid_start, grid_list, grid_big, halton, ocost, stamp,
                       lists, ctl};
        for (void* p : dev)
            if (p) cudaFree(p);
        if (h_ctl) cudaFreeHost(h_ctl);
        if (h_scalars) cudaFreeHost(h_scalars);
        for (auto& pair : ev)
            for (cudaEvent_t e : pair)
                if (e) cudaEventDestroy(e);
    }
};

namespace {

gmt_status check_space(const gmt_space* sp) {
    if (!sp) return fail(GMT_ERR_INVALID, "space is NULL");
    if (sp->kind == GMT_COST_EUCLID) {
        if (sp->dim < 2 || sp->dim > GMT_MAX_DIM || sp->pos_dim != sp->dim)
            return fail(GMT_ERR_INVALID, "Euclidean space needs 2 <= dim <= 10 and pos_dim == dim");
    } else if (sp->kind == GMT_COST_DI) {
        if (sp->dim != 6 || sp->pos_dim != 3)
            return fail(GMT_ERR_INVALID, "double-integrator space needs dim == 6, pos_dim == 3");
    } else if (sp->kind == GMT_COST_DUBINS) {
        if (sp->dim != 4 || sp->pos_dim != 3)
            return fail(GMT_ERR_INVALID, "Dubins airplane space needs dim == 4, pos_dim == 3");
    } else {
        return fail(GMT_ERR_INVALID, "unknown cost kind");
    }
    for (int a = 0; a < sp->dim; ++a)
        if (!(sp->lo[a] < sp->hi[a]) || !std::isfinite(sp->lo[a]) || !std::isfinite(sp->hi[a]))
            return fail(GMT_ERR_INVALID, "state bounds must be finite with lo < hi");
    return GMT_OK;
}

gmt_status check_boxes(const gmt_boxes* b) {
    if (!b) return fail(GMT_ERR_INVALID, "boxes is NULL");
    if (b->count < 0) return fail(GMT_ERR_INVALID, "negative box count");
    if (b->count > 0 && (!b->lo || !b->hi)) return fail(GMT_ERR_INVALID, "box arrays are NULL");
    return GMT_OK;
}

float resolve_radius(const gmt_params* p, int d) {
    if (p->r > 0.0f) return p->r;
    return (float)(p->sampler == GMT_SAMPLER_HALTON ? gmt_connection_radius_halton(p->n, d, p->eta, p->mu_free)
                                                    : gmt_connection_radius(p->n, d, p->eta, p->mu_free));
}

gmt_status check_params(const gmt_params* p, int d) {
    if (!p) return fail(GMT_ERR_INVALID, "params is NULL");
    if (p->n < 1 || p->n > (1 << 24)) return fail(GMT_ERR_INVALID, "n must be in [1, 2^24]");
    if (!(p->lambda >= 0.0f && p->lambda <= 1.0f)) return fail(GMT_ERR_INVALID, "lambda must be in [0, 1]");
    if (p->sampler != GMT_SAMPLER_PHILOX && p->sampler != GMT_SAMPLER_HALTON)
        return fail(GMT_ERR_INVALID, "sampler must be GMT_SAMPLER_PHILOX or GMT_SAMPLER_HALTON");
    if (p->r <= 0.0f && (!(p->eta >= 0.0f) || !(p->mu_free > 0.0f)))
        return fail(GMT_ERR_INVALID, "r <= 0 needs eta >= 0 and mu_free > 0 (Theorem 1 radius)");
    const float r = resolve_radius(p, d);
    if (!(r > 0.0f) || !std::isfinite(r)) return fail(GMT_ERR_INVALID, "connection radius must be positive");
    if (!(p->seg_spacing > 0.0f)) return fail(GMT_ERR_INVALID, "seg_spacing must be positive");
    if (p->traj_points < 2) return fail(GMT_ERR_INVALID, "traj_points must be >= 2");
    return GMT_OK;
}

}  // namespace

extern "C" {

const char* gmt_last_error(void) { return g_last_error.c_str(); }

double gmt_connection_radius_halton(int32_t n, int32_t d, double eta, double mu_free) {
    const double pi = 3.14159265358979323846;
    const double zeta = std::pow(pi, (double)d / 2.0) / std::tgamma((double)d / 2.0 + 1.0);
    const double base = (1.0 + eta) * (1.0 / (double)d) * (mu_free / zeta) * (1.0 / (double)n);
    return 4.0 * std::pow(base, 1.0 / (double)d);
}

double gmt_connection_radius(int32_t n, int32_t d, double eta, double mu_free) {
    const double pi = 3.14159265358979323846;
    const double zeta = std::pow(pi, (double)d / 2.0) / std::tgamma((double)d / 2.0 + 1.0);
    const double base = (1.0 + eta) * (1.0 / (double)d) * (mu_free / zeta) * (std::log((double)n) / (double)n);
    return 4.0 * std::pow(base, 1.0 / (double)d);
}

namespace {
// Box grid over the first two position axes of the graph's space, for at
// least kBoxGridMinBoxes boxes (use = 0 otherwise).
cudaError_t build_box_grid(gmt_graph* g, const BoxArgs& boxes, BoxGridArgs* gr, cudaStream_t st) {
    std::memset(gr, 0, sizeof(*gr));
    if (g->dp < 2 || boxes.count < kBoxGridMinBoxes) return cudaSuccess;
    const int G = box_grid_cells(boxes.count);
    const size_t B = (size_t)boxes.count, cells = (size_t)G * G;
    cudaError_t e;
    if ((e = grow(&g->grid_cnt, &g->cap_grid_cnt, cells + 1)) != cudaSuccess) return e;  // + the big-box count
    if ((e = grow(&g->grid_start, &g->cap_grid_start, cells + 1)) != cudaSuccess) return e;
    if ((e = grow(&g->grid_list, &g->cap_grid_list, B * kBoxGridMaxCells)) != cudaSuccess) return e;
    if ((e = grow(&g->grid_big, &g->cap_grid_big, B)) != cudaSuccess) return e;
    gr->use = 1;
    gr->g = G;
    for (int k = 0; k < 2; ++k) {
        gr->lo[k] = g->pos_lo[k];
        gr->inv_h[k] = (float)((double)G / ((double)g->pos_hi[k] - (double)g->pos_lo[k]));
    }
    gr->start = g->grid_start;
    gr->list = g->grid_list;
    gr->big = g->grid_big;
    gr->nbig = g->grid_cnt + cells;
    if ((e = cudaMemsetAsync(g->grid_cnt, 0, (cells + 1) * sizeof(int), st)) != cudaSuccess) return e;
    return launch_box_grid(g->dp, boxes, *gr, g->grid_cnt, g->grid_start, g->grid_list, g->grid_big,
                           g->grid_cnt + cells, st);
}
}  // namespace

gmt_status gmt_build_graph(const gmt_space* space, const gmt_boxes* boxes, const float* x_init, const gmt_goal* goal,
                           const gmt_params* params, gmt_graph** graph, gmt_stream stream) {
    return gmt_build_graph_ex(space, boxes, x_init, goal, params, nullptr, 0, 0, graph, stream);
}

namespace {
// Edges every edge array of the handle holds now (0 if one is missing).
long long edge_capacity(const gmt_graph* g) {
    long long c = (long long)std::min(g->cap_out_col, g->cap_out_cost);
    if (g->directed()) c = std::min(c, (long long)std::min(g->cap_in_col_own, g->cap_in_cost_own));
    if (g->kind == GMT_COST_DI) c = std::min(c, (long long)std::min(g->cap_out_tau, g->cap_in_tau));
    if (g->kind == GMT_COST_DUBINS) c = std::min(c, (long long)(g->cap_in_path / 4));
    return c;
}

gmt_status build_impl(const gmt_space* space, const gmt_boxes* boxes, const float* x_init, const gmt_goal* goal,
                      const gmt_params* params, const float* extra, int32_t extra_count, int32_t extra_pitch,
                      gmt_graph** graph, gmt_stream stream, bool async);

// Confirms an asynchronous build once its stream has reached the flag and
// edge-count readback: reports sampling errors as the synchronous build does,
// and rebuilds synchronously if the edges outgrew the arrays the fill used.
gmt_status resolve_pending(gmt_graph* g, bool* rebuilt) {
    *rebuilt = false;
    if (!g->pending) return GMT_OK;
    GMT_CUDA(cudaStreamSynchronize(g->pending_stream), "graph build");
    g->pending = false;
    const int flags = g->h_scalars[0];
    g->E = g->h_scalars[2];
    if (flags & kSampleBadInit) return fail(GMT_ERR_INVALID, "x_init is outside X or inside an obstacle");
    if (flags & kSampleExhausted)
        return fail(GMT_ERR_INVALID, "a sample exhausted max_attempts (X_free or X_goal n X_free too small)");
    if (flags & kSampleTimeout) return fail(GMT_ERR_TIMEOUT, "the Halton sampler's bounded wait ran out");
    if (g->E > g->pending_cap) {
        *rebuilt = true;
        gmt_graph* h = g;
        return build_impl(&g->p_space, &g->p_boxes, g->p_x_init, &g->p_goal, &g->p_params, nullptr, 0, 0, &h,
                          (gmt_stream)g->pending_stream, false);
    }
    return GMT_OK;
}
}  // namespace

gmt_status gmt_build_graph_ex(const gmt_space* space, const gmt_boxes* boxes, const float* x_init,
                              const gmt_goal* goal, const gmt_params* params, const float* extra, int32_t extra_count,
                              int32_t extra_pitch, gmt_graph** graph, gmt_stream stream) {
    return build_impl(space, boxes, x_init, goal, params, extra, extra_count, extra_pitch, graph, stream, false);
}

gmt_status gmt_build_graph_async(const gmt_space* space, const gmt_boxes* boxes, const float* x_init,
                                 const gmt_goal* goal, const gmt_params* params, gmt_graph** graph,
                                 gmt_stream stream) {
    return build_impl(space, boxes, x_init, goal, params, nullptr, 0, 0, graph, stream, true);
}

namespace {
gmt_status build_impl(const gmt_space* space, const gmt_boxes* boxes, const float* x_init, const gmt_goal* goal,
                      const gmt_params* params, const float* extra, int32_t extra_count, int32_t extra_pitch,
                      gmt_graph** graph, gmt_stream stream, bool async) {
    gmt_status s;
    if (extra_count < 0 || (extra_count > 0 && (!extra || extra_pitch < extra_count)))
        return fail(GMT_ERR_INVALID, "extra samples need a DEVICE array [dim][extra_pitch], extra_pitch >= count");
    if (extra_count > 0 && space && space->kind == GMT_COST_EUCLID && space->dim > 3)
        return fail(GMT_ERR_INVALID, "appended samples are supported for dim <= 3 and the kinodynamic spaces");
    if ((s = check_space(space)) != GMT_OK) return s;
    if ((s = check_boxes(boxes)) != GMT_OK) return s;
    if ((s = check_params(params, space->dim)) != GMT_OK) return s;
    if (space->kind == GMT_COST_DUBINS &&
        (!(params->turn_radius > 0.0f) || !std::isfinite(params->turn_radius) || !(params->r > 0.0f)))
        return fail(GMT_ERR_INVALID, "a Dubins airplane graph needs turn_radius > 0 and r > 0");
    if (!x_init || !goal || !graph) return fail(GMT_ERR_INVALID, "x_init, goal and graph must be non-NULL");
    if (!(goal->radius >= 0.0f)) return fail(GMT_ERR_INVALID, "goal radius must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;

    const bool fresh = *graph == nullptr;
    gmt_graph* g = fresh ? new gmt_graph() : *graph;
    auto bail = [&](gmt_status st_) {
        if (fresh) delete g;
        return st_;
    };

    g->kind = space->kind;
    g->d = space->dim;
    g->dp = space->pos_dim;
    const int n_sampled = params->n + 1;
    g->N = n_sampled + extra_count;
    g->pitch = (g->N + 31) / 32 * 32;
    g->r = resolve_radius(params, space->dim);
    g->rho = space->kind == GMT_COST_DUBINS ? params->turn_radius : 0.0f;
    g->E = 0;
    for (int a = 0; a < 3 && a < g->dp; ++a) { g->pos_lo[a] = space->lo[a]; g->pos_hi[a] = space->hi[a]; }
    const size_t N = (size_t)g->N, P = (size_t)g->pitch, W = (N + 31) / 32;

    SpaceArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.kind = g->kind; sa.d = g->d; sa.dp = g->dp; sa.N = g->N; sa.pitch = g->pitch;
    sa.n_sampled = n_sampled;
    for (int a = 0; a < g->d; ++a) {
        sa.lo[a] = space->lo[a]; sa.hi[a] = space->hi[a];
        sa.x0[a] = x_init[a]; sa.gc[a] = goal->center[a];
    }
    sa.grho = goal->radius;
    sa.gd = goal->pos_only ? g->dp : g->d;
    sa.key0 = (uint32_t)(params->seed & 0xffffffffu);
    sa.key1 = (uint32_t)(params->seed >> 32);
    sa.stream = 0;
    sa.max_attempts = params->max_attempts > 0 ? params->max_attempts : 65536;
    sa.sampler = params->sampler;
    sa.halton_cap = (long long)sa.max_attempts + 64LL * n_sampled;
    sa.r = g->r;
    sa.r2_threshold = euclid_threshold(g->r);
    sa.rho = g->rho;
    BoxArgs ba{boxes->count, boxes->lo, boxes->hi};

    cudaError_t e;
#define GROW(ptr, n) if ((e = grow(&g->ptr, &g->cap_##ptr, (n))) != cudaSuccess) return bail(cuda_fail(e, "allocating " #ptr))
    GROW(X, (size_t)g->d * P);
    GROW(is_goal, P);
    GROW(out_row, N + 1);
    GROW(counts, kFlagInts + 2 * N);
    g->flags = g->counts;
    g->out_count = g->counts + kFlagInts;
    g->in_count = g->counts + kFlagInts + N;
    GROW(ocost, 2 * (size_t)N);  // two open-set snapshot buffers
    GROW(stamp, N);
    GROW(lists, kPlanListInts * N);
    GROW(ctl, 1);
    if (g->directed()) {
        GROW(in_row_own, N + 1);
        GROW(maskT, W * P);
    }
    // Directed costs (double integrator, Dubins airplane), once earlier builds
    // have sized the edge arrays: the pair filter lists each edge with its cost
    // and arrival time (or shortest word), and the fill places the listed
    // edges by rank instead of solving for them again.
    const bool listed = g->directed() && edge_capacity(g) > 0;
    if (listed) {
        GROW(elist, (size_t)edge_capacity(g));
        if (g->kind == GMT_COST_DUBINS) GROW(epath, (size_t)edge_capacity(g));
        GROW(wpre, W * P);
        GROW(wpreT, W * P);
    }
    size_t list_slots = listed ? g->cap_elist : 0;
    if (listed && g->kind == GMT_COST_DUBINS) list_slots = std::min(list_slots, g->cap_epath);
    const int list_cap = (int)std::min<size_t>(list_slots, (size_t)INT_MAX);
    if (!g->h_ctl && (e = alloc_mapped(&g->h_ctl, &g->d_ctl, 1)) != cudaSuccess)
        return bail(cuda_fail(e, "allocating pinned control block"));
    if (!g->h_scalars && (e = alloc_mapped(&g->h_scalars, &g->d_scalars, 4)) != cudaSuccess)
        return bail(cuda_fail(e, "allocating pinned scalars"));

#define LAUNCH(call, what) if ((e = (call)) != cudaSuccess) return bail(cuda_fail(e, what))
    for (bool& b : g->stage_ran) b = false;
    LAUNCH(cudaMemsetAsync(g->counts, 0, (kFlagInts + (g->directed() ? 2 * N : N)) * sizeof(int), st), "memset");
    LAUNCH(g->mark(gmt_graph::kSample, 0, st), "event");
    BoxGridArgs grid;
    LAUNCH(build_box_grid(g, ba, &grid, st), "box grid kernels");
    void* halton_scratch = nullptr;
    if (sa.sampler == GMT_SAMPLER_HALTON) {
        const size_t bytes = halton_scratch_bytes(sa.halton_cap);
        GROW(halton, bytes / sizeof(int));
        LAUNCH(cudaMemsetAsync(g->halton, 0, bytes, st), "memset");
        LAUNCH(cudaMemsetAsync(g->halton + 1, 0x7f, sizeof(int), st), "memset");  // no chunk has stopped the rest
        halton_scratch = g->halton;
    }
    LAUNCH(launch_sample(sa, ba, grid, halton_scratch, g->X, g->is_goal, g->flags, st), "sample kernel");
    LAUNCH(launch_append(sa, ba, extra, extra_pitch, n_sampled, extra_count, g->X, g->is_goal, g->flags, st),
           "append kernel");
    LAUNCH(g->mark(gmt_graph::kSample, 1, st), "event");
    // neighbour test: cell list for 2D/3D geometric graphs with a small radius
    // (or when forced), else all pairs; both give the same CSR
    CellGrid cg;
    bool cells_pay = false;
    bool cells = make_cell_grid(g->kind, g->d, space->lo, space->hi, g->r, g->N, false, &cg, &cells_pay);
    if (params->debug_flags & GMT_DEBUG_CELLS_LIST) cg.list_only = 1;
    if (params->debug_flags & GMT_DEBUG_PAIRS_ALL) cells = false;
    else if (!(params->debug_flags & GMT_DEBUG_PAIRS_CELLS)) cells = cells && cells_pay;
    // Euclidean graphs of 2 to 4 dimensions fill their CSR by mask tiles
    const bool tiles = fill_tiles_apply(g->kind, g->d, g->N, false);
    LAUNCH(g->mark(gmt_graph::kPair, 0, st), "event");
    if (cells) {
        GROW(cell_of, N);
        GROW(cell_sorted, N);
        GROW(cell_cnt, (size_t)cg.ncells);
        GROW(cell_start, (size_t)cg.ncells + 1);
        LAUNCH(cudaMemsetAsync(g->cell_cnt, 0, (size_t)cg.ncells * sizeof(int), st), "memset");
        LAUNCH(launch_cells_count(sa, g->X, cg, g->cell_of, g->cell_cnt, st), "cell count kernel");
        LAUNCH(launch_scan(g->cell_cnt, g->cell_start, cg.ncells, st), "scan kernel");
        LAUNCH(launch_cells_scatter(g->N, g->cell_of, g->cell_start, g->cell_cnt, g->cell_sorted, st),
               "cell scatter kernel");
        LAUNCH(launch_cells_rows(sa, g->X, cg, g->cell_of, g->cell_start, g->cell_sorted, false, g->out_count,
                                 g->flags + 1, nullptr, nullptr, nullptr, nullptr, st),
               "cell row kernel");
    } else {
        GROW(mask, W * P);
        if (tiles) {
            GROW(tile_cnt, (size_t)fill_tiles_per_row(N) * P);
        }
        // directed costs: the pair filter also writes the transposed matrix
        const bool dir = g->directed();
        LAUNCH(launch_pair_mask(sa, g->X, g->mask, g->out_count, dir ? g->maskT : nullptr,
                                dir ? g->in_count : nullptr, st, tiles ? g->tile_cnt : nullptr,
                                listed ? g->elist : nullptr, g->flags + 5, list_cap,
                                listed && g->kind == GMT_COST_DUBINS ? g->epath : nullptr),
               "pair filter kernel");
    }
    LAUNCH(g->mark(gmt_graph::kPair, 1, st), "event");
    LAUNCH(g->mark(gmt_graph::kScan, 0, st), "event");
    // the scan also stores the sampling flags, the longest cell row and the
    // edge count in the pinned scalars (no copy)
    LAUNCH(launch_scan2(g->out_count, g->out_row, g->directed() ? g->in_count : nullptr,
                        g->directed() ? g->in_row_own : nullptr, g->N, g->flags, g->d_scalars, st,
                        listed ? g->mask : nullptr, g->wpre, listed ? g->maskT : nullptr, g->wpreT, g->pitch),
           "scan kernel");
    LAUNCH(g->mark(gmt_graph::kScan, 1, st), "event");
    g->pending = false;
    const long long cap_now = edge_capacity(g);
    if (async && !cells && extra_count == 0 && cap_now > 0) {
        // no host wait: fill into the arrays of earlier builds; the next plan
        // (or view) confirms the edge count and rebuilds if it did not fit
        const bool di_a = g->kind == GMT_COST_DI, dub_a = g->kind == GMT_COST_DUBINS;
        LAUNCH(g->mark(gmt_graph::kFill, 0, st), "event");
        const FillDir out_dir{g->mask, g->out_row, g->out_col, g->out_cost, di_a ? g->out_tau : nullptr, nullptr,
                              cap_now};
        const FillDir in_dir = g->directed() ? FillDir{g->maskT, g->in_row_own, g->in_col_own, g->in_cost_own,
                                                       di_a ? g->in_tau : nullptr, dub_a ? g->in_path : nullptr,
                                                       cap_now}
                                             : FillDir{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
        if (listed && list_cap >= cap_now) {  // the list holds every edge the arrays can
            LAUNCH(launch_fill_list(sa, g->elist, g->epath, list_cap, out_dir, in_dir, g->wpre, g->wpreT, st),
                   "fill kernel");
        } else if (tiles) {
            LAUNCH(launch_fill_tiles(sa, g->X, out_dir, g->tile_cnt, st), "fill kernel");
        } else {
            LAUNCH(launch_fill(sa, g->X, out_dir, in_dir, g->flags + 3, st), "fill kernel");
        }
        LAUNCH(g->mark(gmt_graph::kFill, 1, st), "event");
        g->used_cells = false;
        g->E = -1;
        g->pending = true;
        g->pending_cap = cap_now;
        g->pending_stream = st;
        g->p_space = *space;
        g->p_boxes = *boxes;
        std::memcpy(g->p_x_init, x_init, space->dim * sizeof(float));
        g->p_goal = *goal;
        g->p_params = *params;
        *graph = g;
        return GMT_OK;
    }
    LAUNCH(cudaStreamSynchronize(st), "graph build");
    if (cells && !cell_fill_fits(cg, g->N, g->h_scalars[1])) {
        // a row too long to sort in shared memory: the all-pairs test instead
        cells = false;
        GROW(mask, W * P);
        if (tiles) {
            GROW(tile_cnt, (size_t)fill_tiles_per_row(N) * P);
        }
        LAUNCH(cudaMemsetAsync(g->out_count, 0, N * sizeof(int), st), "memset");
        LAUNCH(launch_pair_mask(sa, g->X, g->mask, g->out_count, nullptr, nullptr, st, tiles ? g->tile_cnt : nullptr),
               "pair filter kernel");
        LAUNCH(launch_scan(g->out_count, g->out_row, g->N, st), "scan kernel");
        LAUNCH(cudaMemcpyAsync(g->h_scalars + 2, g->out_row + N, sizeof(int), cudaMemcpyDeviceToHost, st),
               "edge count readback");
        LAUNCH(cudaStreamSynchronize(st), "graph build");
    }
    g->used_cells = cells;
    const int flags = g->h_scalars[0];
    if (flags & kSampleBadInit) return bail(fail(GMT_ERR_INVALID, "x_init is outside X or inside an obstacle"));
    if (flags & kSampleExhausted)
        return bail(fail(GMT_ERR_INVALID, "a sample exhausted max_attempts (X_free or X_goal n X_free too small)"));
    if (flags & kSampleBadAppend) return bail(fail(GMT_ERR_INVALID, "an appended sample is outside X or in X_obs"));
    if (flags & kSampleTimeout) return bail(fail(GMT_ERR_TIMEOUT, "the Halton sampler's bounded wait ran out"));
    g->E = g->h_scalars[2];
    const size_t E = (size_t)g->E;
    // edge arrays that have to grow get a quarter of headroom, so that the
    // next asynchronous builds of similar graphs fit them
    const size_t Eg = edge_capacity(g) >= (long long)E ? E : E + E / 4 + 1024;
    GROW(out_col, Eg);
    GROW(out_cost, Eg);
    const bool di = g->kind == GMT_COST_DI, directed = g->directed();
    if (directed) {
        GROW(in_col_own, Eg);
        GROW(in_cost_own, Eg);
    }
    if (di) {
        GROW(out_tau, Eg);
        GROW(in_tau, Eg);
    }
    const bool dubins = g->kind == GMT_COST_DUBINS;
    if (dubins) GROW(in_path, 4 * Eg);
    LAUNCH(g->mark(gmt_graph::kFill, 0, st), "event");
    if (cells) {
        LAUNCH(launch_cells_rows(sa, g->X, cg, g->cell_of, g->cell_start, g->cell_sorted, true, nullptr, nullptr,
                                 g->out_row, g->out_col, g->out_cost, g->flags + 4, st),
               "cell row kernel");
    } else {
        const FillDir out_dir{g->mask, g->out_row, g->out_col, g->out_cost, di ? g->out_tau : nullptr, nullptr, 0};
        const FillDir in_dir = directed ? FillDir{g->maskT, g->in_row_own, g->in_col_own, g->in_cost_own,
                                                  di ? g->in_tau : nullptr, dubins ? g->in_path : nullptr, 0}
                                        : FillDir{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
        if (listed && (long long)E <= (long long)list_cap) {  // the list holds every edge
            LAUNCH(launch_fill_list(sa, g->elist, g->epath, list_cap, out_dir, in_dir, g->wpre, g->wpreT, st),
                   "fill kernel");
        } else if (tiles) {
            LAUNCH(launch_fill_tiles(sa, g->X, out_dir, g->tile_cnt, st), "fill kernel");
        } else {
            LAUNCH(launch_fill(sa, g->X, out_dir, in_dir, g->flags + 3, st), "fill kernel");
        }
    }
    LAUNCH(g->mark(gmt_graph::kFill, 1, st), "event");
#undef GROW
#undef LAUNCH
    *graph = g;
    return GMT_OK;
}

}  // namespace

gmt_status gmt_graph_get_view(const gmt_graph* gc, gmt_graph_view* v) {
    if (!gc || !v) return fail(GMT_ERR_INVALID, "graph and view must be non-NULL");
    gmt_graph* g = const_cast<gmt_graph*>(gc);  // confirming a pending build completes it, nothing else
    bool rebuilt = false;
    const gmt_status ps = resolve_pending(g, &rebuilt);
    if (ps != GMT_OK) return ps;
    v->kind = g->kind; v->dim = g->d; v->pos_dim = g->dp; v->N = g->N; v->x_pitch = g->pitch;
    v->E = g->E; v->r = g->r;
    v->X = g->X; v->is_goal = g->is_goal;
    v->out_row = g->out_row; v->out_col = g->out_col; v->out_cost = g->out_cost;
    v->in_row = g->in_row(); v->in_col = g->in_col(); v->in_cost = g->in_cost();
    v->out_tau = g->kind == GMT_COST_DI ? g->out_tau : nullptr;
    v->in_tau = g->kind == GMT_COST_DI ? g->in_tau : nullptr;
    v->turn_radius = g->rho;
    v->in_path = g->kind == GMT_COST_DUBINS ? g->in_path : nullptr;
    return GMT_OK;
}

void gmt_graph_free(gmt_graph* g) { delete g; }

gmt_status gmt_plan(gmt_graph* g, const gmt_boxes* boxes, const gmt_params* params, int32_t* parent, float* cost,
                    int32_t* path, gmt_plan_info* info, gmt_stream stream) {
    if (!g || g->N == 0) return fail(GMT_ERR_INVALID, "graph is NULL or not built");
    gmt_status s;
    if ((s = check_boxes(boxes)) != GMT_OK) return s;
    if ((s = check_params(params, g->d)) != GMT_OK) return s;
    if (!parent || !cost || !info) return fail(GMT_ERR_INVALID, "parent, cost and info must be non-NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = g->N;

    PlanArgs a;
    std::memset(&a, 0, sizeof(a));
    a.kind = g->kind; a.d = g->d; a.dp = g->dp; a.N = N; a.pitch = g->pitch;
    a.X = g->X; a.is_goal = g->is_goal;
    a.out_row = g->out_row; a.out_col = g->out_col;
    a.in_row = g->in_row(); a.in_col = g->in_col(); a.in_cost = g->in_cost();
    a.in_tau = g->kind == GMT_COST_DI ? g->in_tau : nullptr;
    a.in_path = g->kind == GMT_COST_DUBINS ? g->in_path : nullptr;
    a.boxes = BoxArgs{boxes->count, boxes->lo, boxes->hi};
    a.r = g->r;
    a.delta = params->lambda * g->r;
    a.seg_spacing = params->seg_spacing;
    a.rho = g->rho;
    a.traj_points = params->traj_points;
    a.max_iters = params->max_iters > 0 ? params->max_iters : N + 1;
    a.spin_limit = params->spin_limit;
    a.debug_flags = params->debug_flags;
    a.cost = cost; a.parent = parent; a.path = path;
    a.ocost = g->ocost; a.stamp = g->stamp;
    assign_plan_lists(a, g->lists, (size_t)N);
    a.ctl = g->ctl;
    a.host_ctl = g->d_ctl;  // the kernel leaves its final control block in h_ctl
    for (int k = 0; k < 3; ++k) { a.pos_lo[k] = g->pos_lo[k]; a.pos_hi[k] = g->pos_hi[k]; }
    if (g->pending) {  // an asynchronous build: the kernel reads the CSR only if its edges fit
        a.check_edges = 1;
        a.edge_cap = g->pending_cap;
    }

    int blocks = g->plan_blocks, threads = g->plan_threads, cluster = g->plan_cluster;
    if (blocks <= 0 && cluster <= 0 && threads <= 0 && g->kind == GMT_COST_EUCLID && g->dp == 2 && N <= 2049) {
        // small 2D graphs: one CTA with the wavefront state in shared memory
        // (measured 10-15% faster than a cluster up to about 2k nodes; slower
        // beyond, and for 3D, double-integrator and Dubins graphs, whose
        // iterations carry more work than one SM issues quickly)
        blocks = 1;
        threads = 1024;
    }
    if (blocks <= 0 && cluster <= 0) {
        // automatic: the largest resident thread-block cluster (hardware
        // barriers; measured fastest on GB300 for N from 1e3 to 4e3), else a
        // cooperative grid of one CTA per SM
        if (g->auto_cluster < 0) g->auto_cluster = plan_max_cluster(g->kind, g->dp, N <= 2048 ? 512 : 1024);
        cluster = g->auto_cluster;
        if (threads <= 0) threads = N <= 2048 ? 512 : 1024;
        if (cluster <= 1) blocks = -1;
    }
    if (threads <= 0) threads = 512;
    if (blocks <= 0 && cluster <= 1) blocks = -1;
    if (blocks == 1 && g->plan_threads <= 0) threads = 1024;
    if (cluster <= 1 && (blocks < 0 || blocks > 1)) {
        int dev = 0, sms = 0;
        GMT_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
        GMT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
        const int maxb = plan_max_coresident_blocks(g->kind, g->dp, threads);
        if (maxb <= 0) return fail(GMT_ERR_CUDA, "plan kernel cannot be resident with this block size");
        if (blocks < 0) blocks = sms;
        if (blocks > maxb) blocks = maxb;
    }
    // a cooperative grid's software barrier counts in the control block, which
    // must be zero before its launch; cluster and single-CTA launches clear
    // their result fields themselves
    if (!(cluster > 1 || blocks == 1)) GMT_CUDA(cudaMemsetAsync(g->ctl, 0, sizeof(PlanCtl), st), "memset");
    g->stage_ran[gmt_graph::kPlan] = false;
    GMT_CUDA(g->mark(gmt_graph::kPlan, 0, st), "event");
    // many boxes: bin them on a grid over the first two position axes
    GMT_CUDA(build_box_grid(g, a.boxes, &a.grid, st), "box grid kernels");
    GMT_CUDA(launch_plan(a, blocks, threads, st, cluster), "plan kernel launch");
    GMT_CUDA(g->mark(gmt_graph::kPlan, 1, st), "event");
    g->last_blocks = cluster > 1 ? -cluster : blocks;
    g->last_threads = threads;
    GMT_CUDA(cudaStreamSynchronize(st), "plan kernel");
    if (g->pending) {
        bool rebuilt = false;
        if ((s = resolve_pending(g, &rebuilt)) != GMT_OK) return s;
        if (rebuilt) return gmt_plan(g, boxes, params, parent, cost, path, info, stream);
    }
    const PlanCtl& c = *g->h_ctl;
    std::memset(info, 0, sizeof(*info));
    info->status = c.status;
    info->goal_node = c.goal_node;
    info->path_len = c.path_len;
    info->path_cost = INFINITY;
    if (c.status == GMT_OK && c.goal_node >= 0) {
        unsigned bits = (unsigned)(c.goal_key >> 32);
        std::memcpy(&info->path_cost, &bits, sizeof(float));
    }
    info->iters = c.iters;
    info->final_i = c.final_i;
    info->push_edges = (int64_t)c.push_edges;
    info->pull_edges = (int64_t)c.pull_edges;
    info->checks = (int64_t)c.checks;
    info->failed = (int64_t)c.failed;
    info->tree_size = (int64_t)c.tree_size;
    if (c.status == GMT_ERR_TIMEOUT) return fail(GMT_ERR_TIMEOUT, "a device-side wait ran out (spin limit)");
    if (c.status == GMT_ERR_ITER_LIMIT) return fail(GMT_ERR_ITER_LIMIT, "group expansions exceeded max_iters");
    return (gmt_status)c.status;
}

gmt_status gmt_graph_set_profiling(gmt_graph* g, int32_t enable) {
    if (!g) return fail(GMT_ERR_INVALID, "graph is NULL");
    if (enable < 0 || enable > 2) return fail(GMT_ERR_INVALID, "profiling must be 0, 1 or 2");
    g->profiling = enable;
    return GMT_OK;
}

gmt_status gmt_graph_get_profile(gmt_graph* g, gmt_profile* out) {
    if (!g || !out) return fail(GMT_ERR_INVALID, "graph and profile must be non-NULL");
    float ms[gmt_graph::kStages] = {};
    for (int k = 0; k < gmt_graph::kStages; ++k) {
        if (!g->stage_ran[k] || !g->ev[k][0] || !g->ev[k][1]) continue;
        GMT_CUDA(cudaEventSynchronize(g->ev[k][1]), "profile event");
        GMT_CUDA(cudaEventElapsedTime(&ms[k], g->ev[k][0], g->ev[k][1]), "profile event");
    }
    out->sample_ms = ms[gmt_graph::kSample];
    out->pair_ms = ms[gmt_graph::kPair];
    out->transpose_ms = ms[gmt_graph::kTranspose];
    out->scan_ms = ms[gmt_graph::kScan];
    out->fill_ms = ms[gmt_graph::kFill];
    out->plan_ms = ms[gmt_graph::kPlan];
    out->plan_blocks = g->last_blocks;
    out->plan_threads = g->last_threads;
    return GMT_OK;
}

gmt_status gmt_graph_set_launch(gmt_graph* g, int32_t blocks, int32_t threads, int32_t cluster) {
    if (!g) return fail(GMT_ERR_INVALID, "graph is NULL");
    if (threads != 0 && (threads < 64 || threads > 1024 || threads % 32 != 0))
        return fail(GMT_ERR_INVALID, "threads must be 0 or a multiple of 32 in [64, 1024]");
    if (blocks < 0) return fail(GMT_ERR_INVALID, "blocks must be >= 0");
    if (cluster < 0 || cluster > 16) return fail(GMT_ERR_INVALID, "cluster must be in [0, 16]");
    g->plan_blocks = blocks;
    g->plan_threads = threads;
    g->plan_cluster = cluster;
    return GMT_OK;
}

}  // extern "C"
