// gmt_plan_static: the wavefront of gmt_plan without any device allocation.
//
// Some callers cannot allocate device memory when they plan: a replanning
// loop inside a control cycle (a cudaMalloc or cudaFree may synchronise the
// whole device and has no latency bound), or systems that fix their memory at
// start-up.  This entry point takes the graph as plain device arrays (a
// gmt_graph_view the caller fills) and runs the same plan kernel as gmt_plan;
// the kernel's scratch (open-set snapshot, claim stamps, group/open/candidate
// lists, control block and barrier words) lives in one file-scope __device__
// array of fixed size instead of being allocated.
//
//  - Capacity: graphs of at most GMT_STATIC_MAX_NODES nodes; larger ones are
//    rejected with GMT_ERR_INVALID.  The array takes about 2.6 MB on every GPU
//    that loads the library, for the life of the process.
//  - Set-up: the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress, with that device current) and caches it, together
//    with the largest resident cluster of the plan kernel; make that first
//    call before any stream capture begins.
//  - Launch: the same automatic shape as gmt_plan (one CTA with its state in
//    shared memory for small 2D graphs, else the largest resident thread-block
//    cluster, else a cooperative grid).  Obstacles are scanned linearly by
//    every check: the box grid that gmt_plan builds for 128 or more boxes needs
//    allocated scratch, so many boxes cost more here than in gmt_plan.
//  - Sharing: every call on a device uses the same array and the array keeps
//    the last call's contents; the control block is cleared at the start of
//    each call.  Calls whose kernels overlap on the GPU (other streams, other
//    host threads) race on the array: serialise them.
//  - No cudaMalloc, cudaFree or allocating library routine is called.
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

using namespace gmtk;

namespace {

constexpr size_t kCtlSlot = 256;
static_assert(sizeof(PlanCtl) <= kCtlSlot, "control block must fit its slot");
constexpr size_t kNodes = GMT_STATIC_MAX_NODES;
// [control block][ocost: 2 kNodes floats (two snapshot buffers)][stamp: kNodes ints]
// [lists: kPlanListInts kNodes ints]
constexpr size_t kScratchBytes =
    kCtlSlot + 2 * kNodes * sizeof(float) + kNodes * sizeof(int) + (size_t)kPlanListInts * kNodes * sizeof(int);

static __device__ __align__(256) unsigned char g_plan_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};
// plan_max_cluster per device and kernel (double integrator, Dubins, 2D, other
// geometric) x threads (512, 1024); -1 = not probed yet
int g_cluster[kMaxDevices][4][2];
bool g_cluster_init = false;

gmt_status fail(gmt_status s, const std::string& m) {
    record_error(m.c_str());  // readable through gmt_last_error()
    return s;
}

gmt_status cuda_fail(cudaError_t e, const char* what) {
    return fail(GMT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Device address of the scratch array on the current device (looked up once).
gmt_status scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(GMT_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_plan_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_addr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_addr[dev];
    return GMT_OK;
}

// Largest resident cluster of the plan kernel on the current device (cached).
gmt_status max_cluster(int kind, int dp, int threads, int* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(GMT_ERR_INVALID, "device index out of range");
    const int k = kind == GMT_COST_DI ? 0 : kind == GMT_COST_DUBINS ? 1 : dp == 2 ? 2 : 3;
    const int t = threads == 1024 ? 1 : 0;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_cluster_init) {
        for (auto& d : g_cluster)
            for (auto& kk : d)
                for (int& v : kk) v = -1;
        g_cluster_init = true;
    }
    if (g_cluster[dev][k][t] < 0) g_cluster[dev][k][t] = plan_max_cluster(kind, dp, threads);
    *out = g_cluster[dev][k][t];
    return GMT_OK;
}

}  // namespace

extern "C" gmt_status gmt_plan_static(const gmt_space* space, const gmt_graph_view* g, const gmt_boxes* boxes,
                                      const gmt_params* params, int32_t* parent, float* cost, int32_t* path,
                                      gmt_plan_info* info, gmt_stream stream) {
    if (!space || !g || !boxes || !params || !parent || !cost || !info)
        return fail(GMT_ERR_INVALID, "space, graph, boxes, params, parent, cost and info must be non-NULL");
    if (g->N < 1 || g->N > GMT_STATIC_MAX_NODES)
        return fail(GMT_ERR_INVALID, "gmt_plan_static: graph has " + std::to_string(g->N) +
                                         " nodes; the static scratch holds at most " +
                                         std::to_string(GMT_STATIC_MAX_NODES));
    if (g->kind != space->kind || g->dim != space->dim || g->pos_dim != space->pos_dim)
        return fail(GMT_ERR_INVALID, "graph view and space disagree on kind or dimensions");
    if (g->kind != GMT_COST_EUCLID && g->kind != GMT_COST_DI && g->kind != GMT_COST_DUBINS)
        return fail(GMT_ERR_INVALID, "unknown cost kind");
    if (g->kind == GMT_COST_DI       ? (g->dim != 6 || g->pos_dim != 3)
        : g->kind == GMT_COST_DUBINS ? (g->dim != 4 || g->pos_dim != 3 || !(g->turn_radius > 0.0f))
                                     : (g->dim < 2 || g->dim > GMT_MAX_DIM || g->pos_dim != g->dim))
        return fail(GMT_ERR_INVALID, "unsupported dimensions (or a Dubins view without a turning radius)");
    if (g->x_pitch < g->N || g->E < 0 || !g->X || !g->is_goal || !g->out_row || !g->in_row ||
        (g->E > 0 && (!g->out_col || !g->in_col || !g->in_cost)))
        return fail(GMT_ERR_INVALID, "graph view has missing arrays or a bad pitch");
    if (!(g->r > 0.0f)) return fail(GMT_ERR_INVALID, "graph radius must be positive");
    if (boxes->count < 0 || (boxes->count > 0 && (!boxes->lo || !boxes->hi)))
        return fail(GMT_ERR_INVALID, "bad box arrays");
    if (!(params->lambda >= 0.0f && params->lambda <= 1.0f)) return fail(GMT_ERR_INVALID, "lambda must be in [0, 1]");
    if (!(params->seg_spacing > 0.0f) || params->traj_points < 2)
        return fail(GMT_ERR_INVALID, "seg_spacing must be > 0 and traj_points >= 2");

    unsigned char* base = nullptr;
    gmt_status s = scratch_address(&base);
    if (s != GMT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t NM = kNodes;
    PlanCtl* ctl = (PlanCtl*)base;
    float* ocost = (float*)(base + kCtlSlot);
    int* stamp = (int*)(base + kCtlSlot + 2 * NM * sizeof(float));
    int* lists = stamp + NM;

    PlanArgs a;
    std::memset(&a, 0, sizeof(a));
    a.kind = g->kind; a.d = g->dim; a.dp = g->pos_dim; a.N = g->N; a.pitch = g->x_pitch;
    a.X = g->X; a.is_goal = g->is_goal;
    a.out_row = g->out_row; a.out_col = g->out_col;
    a.in_row = g->in_row; a.in_col = g->in_col; a.in_cost = g->in_cost;
    a.in_tau = g->kind == GMT_COST_DI ? g->in_tau : nullptr;
    a.in_path = g->kind == GMT_COST_DUBINS ? g->in_path : nullptr;
    a.boxes = BoxArgs{boxes->count, boxes->lo, boxes->hi};
    for (int k = 0; k < 3 && k < g->pos_dim; ++k) { a.pos_lo[k] = space->lo[k]; a.pos_hi[k] = space->hi[k]; }
    a.r = g->r;
    a.delta = params->lambda * g->r;
    a.seg_spacing = params->seg_spacing;
    a.rho = g->kind == GMT_COST_DUBINS ? g->turn_radius : 0.0f;
    a.traj_points = params->traj_points;
    a.max_iters = params->max_iters > 0 ? params->max_iters : g->N + 1;
    a.spin_limit = params->spin_limit;
    a.debug_flags = params->debug_flags;
    a.cost = cost; a.parent = parent; a.path = path;
    a.ocost = ocost; a.stamp = stamp;
    assign_plan_lists(a, lists, NM);
    a.ctl = ctl;

    // launch shape: as gmt_plan chooses it automatically
    int blocks = 0, cluster = 0, threads = 0;
    if (g->kind == GMT_COST_EUCLID && g->pos_dim == 2 && g->N <= 2049) {
        blocks = 1;  // one CTA, wavefront state in shared memory
        threads = 1024;
    } else {
        threads = g->N <= 2048 ? 512 : 1024;
        s = max_cluster(g->kind, g->pos_dim, threads, &cluster);
        if (s != GMT_OK) return s;
        if (cluster <= 1) {
            cluster = 0;
            int dev = 0, sms = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return cuda_fail(e, "device attribute");
            const int maxb = plan_max_coresident_blocks(g->kind, g->pos_dim, threads);
            if (maxb <= 0) return fail(GMT_ERR_CUDA, "plan kernel cannot be resident");
            blocks = sms < maxb ? sms : maxb;
        }
    }
    // a cooperative grid's barrier counts live in the control block and must
    // start at zero; the other launches clear their result fields themselves
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(PlanCtl), st);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the control block");
    e = launch_plan(a, blocks, threads, st, cluster);
    if (e != cudaSuccess) return cuda_fail(e, "plan kernel launch");
    PlanCtl c;
    e = cudaMemcpyAsync(&c, ctl, sizeof(PlanCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "plan kernel");

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
    if (c.status == GMT_ERR_TIMEOUT) return fail(GMT_ERR_TIMEOUT, "a device-side wait ran out (spin limit)");
    if (c.status == GMT_ERR_ITER_LIMIT) return fail(GMT_ERR_ITER_LIMIT, "group expansions exceeded max_iters");
    return (gmt_status)c.status;
}
