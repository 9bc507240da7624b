// Replanning server (gmt_server_*): a continuous-batching request loop around
// the wavefront kernel.
//
// Sessions keep their samples and neighbour CSR resident on the device: the
// connection costs do not depend on the obstacles, so only the collision
// verdicts can change when boxes move.  Each session also keeps a cache of
// per-edge verdicts and, per edge, the bounding box of the points its check
// tests; before a request is planned, the entries whose bounding box touches
// the old or the new place of a moved box are cleared, so only edges near
// moved obstacles are checked again.  Plans on stale-free caches are identical
// to fresh plans (tested).
//
// Requests are queued on the host; a worker thread admits the oldest request
// of an idle session to any free slot (a CUDA stream with its own plan
// scratch) as soon as one frees up, so requests that arrive while others run
// overlap on the device.  Sessions are admitted against a device-memory budget
// (GMT_ERR_ADMISSION when they do not fit).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gmtk {

// Bounding box (over the position axes) of the points the lazy check of in-edge
// e tests: the m segment points (geometric), the trajectory points (double
// integrator) or the points along the stored shortest word (Dubins airplane),
// computed with the same expressions as the check.
template <int KIND, int DP>
__global__ void edge_aabb_kernel(int N, int pitch, const float* __restrict__ X, const int* __restrict__ in_row,
                                 const int* __restrict__ in_col, const float* __restrict__ in_cost,
                                 const float* __restrict__ in_tau, const float* __restrict__ in_path, float rho,
                                 float seg_spacing, int traj_points, float* __restrict__ aabb) {
    const int x = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (x >= N) return;
    constexpr int D = KIND == GMT_COST_DI ? 6 : (KIND == GMT_COST_DUBINS ? 4 : DP);
    constexpr int P = KIND == GMT_COST_EUCLID ? DP : 3;
    float sx[D];
#pragma unroll
    for (int a = 0; a < D; ++a) sx[a] = X[(size_t)a * pitch + x];
    for (int e = in_row[x] + lane; e < in_row[x + 1]; e += 32) {
        const int y = in_col[e];
        float sy[D];
#pragma unroll
        for (int a = 0; a < D; ++a) sy[a] = X[(size_t)a * pitch + y];
        float lo[P], hi[P];
#pragma unroll
        for (int a = 0; a < P; ++a) { lo[a] = f_inf(); hi[a] = -f_inf(); }
        if (KIND == GMT_COST_DUBINS) {
            const float4 w = reinterpret_cast<const float4*>(in_path)[e];
            const DubPath Pw{__float_as_int(w.w), w.x, w.y, w.z, ((w.x + w.y) + w.z) * rho};
            if (Pw.word < kDubNone) {
                const DubSegs G = dubins_segments(sy, Pw, rho);
                int m = (int)ceilf(in_cost[e] / seg_spacing) + 1;
                if (m < 2) m = 2;
                const float denom = (float)(m - 1);
                for (int k = 0; k < m; ++k) {
                    float p[3];
                    dubins_point(sy, sx, G, (float)k / denom, p);
#pragma unroll
                    for (int a = 0; a < P; ++a) { lo[a] = fminf(lo[a], p[a]); hi[a] = fmaxf(hi[a], p[a]); }
                }
            }
        } else if (KIND == GMT_COST_EUCLID) {
            int m = (int)ceilf(in_cost[e] / seg_spacing) + 1;
            if (m < 2) m = 2;
            const float denom = (float)(m - 1);
            for (int k = 0; k < m; ++k) {
                const float t = (float)k / denom;
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const float p = sy[a] + t * (sx[a] - sy[a]);
                    lo[a] = fminf(lo[a], p); hi[a] = fmaxf(hi[a], p);
                }
            }
        } else {
            const float tau = in_tau[e];
            const float denom = (float)(traj_points - 1);
            for (int k = 0; k < traj_points; ++k) {
                float p[3];
                hermite_point(sy, sx, tau, (float)k / denom, p);
#pragma unroll
                for (int a = 0; a < P; ++a) { lo[a] = fminf(lo[a], p[a]); hi[a] = fmaxf(hi[a], p[a]); }
            }
        }
#pragma unroll
        for (int a = 0; a < P; ++a) {
            aabb[(size_t)e * 2 * P + a] = lo[a];
            aabb[(size_t)e * 2 * P + P + a] = hi[a];
        }
    }
}

// Clears the cached verdict of every edge whose point box meets one of the
// `nm` moved-box regions (their old and new places, [nm][2][P] lo/hi pairs).
template <int P>
__global__ void invalidate_kernel(long long E, const float* __restrict__ aabb, const float* __restrict__ moved,
                                  int nm, uint8_t* __restrict__ verdict) {
    extern __shared__ float mv[];
    for (int t = threadIdx.x; t < nm * 4 * P; t += blockDim.x) mv[t] = moved[t];
    __syncthreads();
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E || verdict[e] == 0) return;
    float lo[P], hi[P];
#pragma unroll
    for (int a = 0; a < P; ++a) { lo[a] = aabb[e * 2 * P + a]; hi[a] = aabb[e * 2 * P + P + a]; }
    for (int k = 0; k < 2 * nm; ++k) {
        const float* b = mv + k * 2 * P;
        bool meet = true;
#pragma unroll
        for (int a = 0; a < P; ++a) meet = meet && lo[a] <= b[P + a] && b[a] <= hi[a];
        if (meet) { verdict[e] = 0; return; }
    }
}

}  // namespace gmtk

using namespace gmtk;

namespace {

using Clock = std::chrono::steady_clock;

struct Session {
    int id = 0;
    gmt_space space;
    gmt_goal goal;
    gmt_params params;
    float x_init[GMT_MAX_DIM] = {};
    gmt_graph* graph = nullptr;
    gmt_graph_view view;
    int nbox = 0, dp = 0;
    std::vector<float> cur_lo, cur_hi;  // boxes the cache is valid for
    float* d_lo = nullptr;
    float* d_hi = nullptr;
    float* aabb = nullptr;
    uint8_t* verdict = nullptr;
    size_t bytes = 0;
    bool busy = false;
    bool closing = false;
    bool moving = false;  // a start move is rebuilding the graph: requests wait in the queue
};

struct Request {
    uint64_t id = 0;
    int session = 0;
    std::vector<float> lo, hi;
    int32_t* parent = nullptr;
    float* cost = nullptr;
    Clock::time_point t_submit;
};

struct Slot {
    std::condition_variable* cv = nullptr;  // server's, notified when the slot's request finishes
    cudaStream_t stream = nullptr;
    float* ocost = nullptr;
    int* stamp = nullptr;
    int* lists = nullptr;
    PlanCtl* ctl = nullptr;
    int32_t* parent = nullptr;
    float* cost = nullptr;
    float* moved = nullptr;       // device [2 * max_boxes][2][3]
    float* h_moved = nullptr;     // pinned staging
    float* h_boxes = nullptr;     // pinned staging of the request's boxes
    PlanCtl* h_ctl = nullptr;
    bool busy = false;
    std::atomic<int> finished{0};
    Request req;
    Clock::time_point t_start, t_done;
};

}  // namespace

struct gmt_server {
    gmt_server_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::vector<std::unique_ptr<Slot>> slots;
    std::map<int, Session> sessions;
    std::vector<gmt_server_result> done;
    std::thread worker;
    bool stop = false;
    int next_session = 1;
    size_t used_bytes = 0;
    std::string worker_error;
    cudaStream_t setup = nullptr;
};

namespace {

gmt_status sfail(gmt_status s, const std::string& m) {
    record_error(m.c_str());
    return s;
}

void CUDART_CB on_done(void* p) {
    Slot* s = (Slot*)p;
    s->t_done = Clock::now();
    s->finished.store(1);
    s->cv->notify_all();
}

// Launches a request on a free slot (worker thread, server lock held).
cudaError_t start_request(gmt_server* sv, Slot& sl, Session& ss, Request&& rq) {
    const int P = ss.dp, nb = ss.nbox;
    sl.req = std::move(rq);
    sl.t_start = Clock::now();
    sl.finished.store(0);
    cudaStream_t st = sl.stream;
    // moved boxes: old and new places of every box that changed
    int nm = 0;
    for (int b = 0; b < nb; ++b) {
        bool moved = false;
        for (int a = 0; a < P; ++a)
            moved = moved || sl.req.lo[b * P + a] != ss.cur_lo[b * P + a] || sl.req.hi[b * P + a] != ss.cur_hi[b * P + a];
        if (!moved) continue;
        float* o = sl.h_moved + (size_t)nm * 4 * P;
        for (int a = 0; a < P; ++a) {
            o[a] = ss.cur_lo[b * P + a]; o[P + a] = ss.cur_hi[b * P + a];
            o[2 * P + a] = sl.req.lo[b * P + a]; o[3 * P + a] = sl.req.hi[b * P + a];
        }
        ++nm;
    }
    std::memcpy(sl.h_boxes, sl.req.lo.data(), nb * P * sizeof(float));
    std::memcpy(sl.h_boxes + nb * P, sl.req.hi.data(), nb * P * sizeof(float));
    cudaError_t e = cudaSuccess;
    if (nb > 0) {
        e = cudaMemcpyAsync(ss.d_lo, sl.h_boxes, nb * P * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ss.d_hi, sl.h_boxes + nb * P, nb * P * sizeof(float), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && nm > 0 && ss.view.E > 0) {
        e = cudaMemcpyAsync(sl.moved, sl.h_moved, (size_t)nm * 4 * P * sizeof(float), cudaMemcpyHostToDevice, st);
        const long long E = ss.view.E;
        const unsigned blocks = (unsigned)((E + 255) / 256);
        const size_t smem = (size_t)nm * 4 * P * sizeof(float);
        if (e == cudaSuccess) {
            if (P == 3) invalidate_kernel<3><<<blocks, 256, smem, st>>>(E, ss.aabb, sl.moved, nm, ss.verdict);
            else invalidate_kernel<2><<<blocks, 256, smem, st>>>(E, ss.aabb, sl.moved, nm, ss.verdict);
            e = cudaGetLastError();
        }
    }
    ss.cur_lo = sl.req.lo;
    ss.cur_hi = sl.req.hi;
    if (e != cudaSuccess) return e;
    const gmt_graph_view& v = ss.view;
    PlanArgs a;
    std::memset(&a, 0, sizeof(a));
    a.kind = v.kind; a.d = v.dim; a.dp = v.pos_dim; a.N = v.N; a.pitch = v.x_pitch;
    a.X = v.X; a.is_goal = v.is_goal; a.out_row = v.out_row; a.out_col = v.out_col;
    a.in_row = v.in_row; a.in_col = v.in_col; a.in_cost = v.in_cost; a.in_tau = v.in_tau;
    a.in_path = v.in_path;
    a.rho = v.turn_radius;
    a.boxes = BoxArgs{nb, ss.d_lo, ss.d_hi};
    for (int k = 0; k < 3 && k < v.pos_dim; ++k) { a.pos_lo[k] = ss.space.lo[k]; a.pos_hi[k] = ss.space.hi[k]; }
    a.r = v.r;
    a.delta = ss.params.lambda * v.r;
    a.seg_spacing = ss.params.seg_spacing;
    a.traj_points = ss.params.traj_points;
    a.max_iters = ss.params.max_iters > 0 ? ss.params.max_iters : v.N + 1;
    a.spin_limit = ss.params.spin_limit;
    a.cost = sl.req.cost ? sl.req.cost : sl.cost;
    a.parent = sl.req.parent ? sl.req.parent : sl.parent;
    a.ocost = sl.ocost; a.stamp = sl.stamp;
    const size_t M = (size_t)sv->cfg.max_nodes;
    assign_plan_lists(a, sl.lists, M);
    a.ctl = sl.ctl;
    a.verdict = ss.verdict;
    e = cudaMemsetAsync(sl.ctl, 0, sizeof(PlanCtl), st);
    if (e == cudaSuccess)
        e = launch_plan(a, sv->cfg.cluster > 1 ? 0 : 1, sv->cfg.threads, st, sv->cfg.cluster > 1 ? sv->cfg.cluster : 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_ctl, sl.ctl, sizeof(PlanCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_done, &sl);
    return e;
}

void worker_loop(gmt_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        bool progress = false;
        for (auto& up : sv->slots) {
            Slot& sl = *up;
            if (!sl.busy || !sl.finished.load()) continue;
            const PlanCtl& c = *sl.h_ctl;
            gmt_server_result r;
            std::memset(&r, 0, sizeof(r));
            r.request_id = sl.req.id;
            r.session = sl.req.session;
            r.status = c.status;
            r.goal_node = c.goal_node;
            r.path_cost = INFINITY;
            if (c.status == GMT_OK && c.goal_node >= 0) {
                const unsigned bits = (unsigned)(c.goal_key >> 32);
                std::memcpy(&r.path_cost, &bits, sizeof(float));
            }
            r.iters = c.iters;
            r.checks = (int64_t)c.checks;
            r.checks_computed = (int64_t)c.checks_computed;
            r.edges_checked = (int64_t)(c.push_edges + c.pull_edges);
            r.queue_ms = std::chrono::duration<double, std::milli>(sl.t_start - sl.req.t_submit).count();
            r.latency_ms = std::chrono::duration<double, std::milli>(sl.t_done - sl.req.t_submit).count();
            sv->done.push_back(r);
            auto it = sv->sessions.find(sl.req.session);
            if (it != sv->sessions.end()) it->second.busy = false;
            sl.busy = false;
            progress = true;
        }
        for (auto& up : sv->slots) {
            Slot& sl = *up;
            if (sl.busy) continue;
            auto qit = std::find_if(sv->queue.begin(), sv->queue.end(), [&](const Request& q) {
                auto s = sv->sessions.find(q.session);
                return s != sv->sessions.end() && !s->second.busy && !s->second.moving;
            });
            if (qit == sv->queue.end()) break;
            Session& ss = sv->sessions[qit->session];
            Request rq = std::move(*qit);
            sv->queue.erase(qit);
            ss.busy = true;
            sl.busy = true;
            cudaError_t e = start_request(sv, sl, ss, std::move(rq));
            if (e != cudaSuccess) {
                sv->worker_error = std::string("request launch: ") + cudaGetErrorString(e);
                gmt_server_result r;
                std::memset(&r, 0, sizeof(r));
                r.request_id = sl.req.id;
                r.session = sl.req.session;
                r.status = GMT_ERR_CUDA;
                r.path_cost = INFINITY;
                sv->done.push_back(r);
                ss.busy = false;
                sl.busy = false;
            }
            progress = true;
        }
        if (progress) sv->cv.notify_all();
        bool any_busy = false;
        for (auto& up : sv->slots) any_busy = any_busy || up->busy;
        if (!progress) sv->cv.wait_for(lk, any_busy ? std::chrono::microseconds(200) : std::chrono::milliseconds(2));
    }
}

size_t session_bytes_estimate(int N, int kind) {
    const size_t P = (size_t)(N + 31) / 32 * 32, W = (size_t)(N + 31) / 32;
    const size_t E = (size_t)N * 256;  // upper estimate of edges per node
    // bit matrices (and, for directed costs, the transpose and both matrices'
    // word prefixes of a rebuild that places listed edges)
    const size_t mask = W * P * 4 * (kind == GMT_COST_EUCLID ? 1 : 4);
    // per edge: CSR columns and costs (both directions for directed costs),
    // arrival times (DI) or stored words (Dubins), point box, verdict, and the
    // pair filter's edge list of a rebuild (16 B, and 16 B of words for Dubins)
    return mask + E * (kind == GMT_COST_DI ? 60 : kind == GMT_COST_DUBINS ? 89 : 33) + (size_t)N * 64;
}

}  // namespace

extern "C" {

gmt_status gmt_server_create(const gmt_server_config* cfg, gmt_server** out) {
    if (!cfg || !out) return sfail(GMT_ERR_INVALID, "config and out must be non-NULL");
    if (cfg->slots < 1 || cfg->slots > 256 || cfg->max_nodes < 2 || cfg->max_boxes < 0 || cfg->cluster < 0 ||
        cfg->cluster > 16 || (cfg->threads != 0 && (cfg->threads < 64 || cfg->threads > 1024 || cfg->threads % 32)))
        return sfail(GMT_ERR_INVALID, "server config out of range");
    gmt_server* sv = new gmt_server();
    sv->cfg = *cfg;
    if (sv->cfg.threads == 0) sv->cfg.threads = sv->cfg.cluster > 1 ? 512 : 1024;
    cudaGetDevice(&sv->device);
    const size_t M = (size_t)cfg->max_nodes;
    const int mb = std::max(1, cfg->max_boxes);
    cudaError_t e = cudaStreamCreateWithFlags(&sv->setup, cudaStreamNonBlocking);
    for (int k = 0; k < cfg->slots && e == cudaSuccess; ++k) {
        auto sl = std::make_unique<Slot>();
        sl->cv = &sv->cv;
        e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&sl->ocost, 2 * M * 4);  // two snapshot buffers
        if (e == cudaSuccess) e = cudaMalloc(&sl->stamp, M * 4);
        if (e == cudaSuccess) e = cudaMalloc(&sl->lists, M * kPlanListInts * 4);
        if (e == cudaSuccess) e = cudaMalloc(&sl->ctl, 256);
        if (e == cudaSuccess) e = cudaMalloc(&sl->parent, M * 4);
        if (e == cudaSuccess) e = cudaMalloc(&sl->cost, M * 4);
        if (e == cudaSuccess) e = cudaMalloc(&sl->moved, (size_t)mb * 4 * 3 * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&sl->h_moved, (size_t)mb * 4 * 3 * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&sl->h_boxes, (size_t)mb * 2 * 3 * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&sl->h_ctl, sizeof(PlanCtl));
        sv->slots.push_back(std::move(sl));
    }
    if (e != cudaSuccess) {
        gmt_server_free(sv);
        return sfail(e == cudaErrorMemoryAllocation ? GMT_ERR_OOM : GMT_ERR_CUDA,
                     std::string("server allocation: ") + cudaGetErrorString(e));
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return GMT_OK;
}

void gmt_server_free(gmt_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (auto& up : sv->slots) {
        Slot& sl = *up;
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        void* d[] = {sl.ocost, sl.stamp, sl.lists, sl.ctl, sl.parent, sl.cost, sl.moved};
        for (void* p : d)
            if (p) cudaFree(p);
        if (sl.h_moved) cudaFreeHost(sl.h_moved);
        if (sl.h_boxes) cudaFreeHost(sl.h_boxes);
        if (sl.h_ctl) cudaFreeHost(sl.h_ctl);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (auto& kv : sv->sessions) {
        Session& s = kv.second;
        gmt_graph_free(s.graph);
        void* d[] = {s.d_lo, s.d_hi, s.aabb, s.verdict};
        for (void* p : d)
            if (p) cudaFree(p);
    }
    if (sv->setup) cudaStreamDestroy(sv->setup);
    delete sv;
}

namespace {
// Allocates and fills a session's per-edge point boxes and clears its verdict
// cache (all unknown) for the graph `v`.
cudaError_t edge_cache_setup(const gmt_graph_view& v, const gmt_space& space, const gmt_params& params, float** aabb,
                             uint8_t** verdict, cudaStream_t st) {
    const long long E = v.E;
    const int P = space.pos_dim;
    cudaError_t e = cudaMalloc(aabb, std::max(1ll, E) * 2 * P * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(verdict, std::max(1ll, E));
    if (e == cudaSuccess) e = cudaMemsetAsync(*verdict, 0, std::max(1ll, E), st);
    if (e == cudaSuccess && E > 0) {
        const unsigned blocks = (unsigned)((v.N + 7) / 8);
        if (space.kind == GMT_COST_DI)
            edge_aabb_kernel<GMT_COST_DI, 3><<<blocks, 256, 0, st>>>(
                v.N, v.x_pitch, v.X, v.in_row, v.in_col, v.in_cost, v.in_tau, nullptr, 0.0f, params.seg_spacing,
                params.traj_points, *aabb);
        else if (space.kind == GMT_COST_DUBINS)
            edge_aabb_kernel<GMT_COST_DUBINS, 3><<<blocks, 256, 0, st>>>(
                v.N, v.x_pitch, v.X, v.in_row, v.in_col, v.in_cost, nullptr, v.in_path, v.turn_radius,
                params.seg_spacing, params.traj_points, *aabb);
        else if (space.dim == 2)
            edge_aabb_kernel<GMT_COST_EUCLID, 2><<<blocks, 256, 0, st>>>(
                v.N, v.x_pitch, v.X, v.in_row, v.in_col, v.in_cost, nullptr, nullptr, 0.0f, params.seg_spacing,
                params.traj_points, *aabb);
        else
            edge_aabb_kernel<GMT_COST_EUCLID, 3><<<blocks, 256, 0, st>>>(
                v.N, v.x_pitch, v.X, v.in_row, v.in_col, v.in_cost, nullptr, nullptr, 0.0f, params.seg_spacing,
                params.traj_points, *aabb);
        e = cudaGetLastError();
    }
    return e;
}
}  // namespace

gmt_status gmt_server_open_session(gmt_server* sv, const gmt_space* space, const float* x_init, const gmt_goal* goal,
                                   const gmt_params* params, int32_t box_count, const float* box_lo,
                                   const float* box_hi, int32_t* session) {
    if (!sv || !space || !x_init || !goal || !params || !session || box_count < 0 ||
        (box_count > 0 && (!box_lo || !box_hi)))
        return sfail(GMT_ERR_INVALID, "bad session arguments");
    if (box_count > sv->cfg.max_boxes) return sfail(GMT_ERR_INVALID, "more boxes than the server's max_boxes");
    if (params->n + 1 > sv->cfg.max_nodes) return sfail(GMT_ERR_INVALID, "more nodes than the server's max_nodes");
    if (!(space->kind == GMT_COST_DI || space->kind == GMT_COST_DUBINS ||
          (space->kind == GMT_COST_EUCLID && (space->dim == 2 || space->dim == 3))))
        return sfail(GMT_ERR_INVALID,
                     "sessions support the double integrator, the Dubins airplane and 2D/3D geometric spaces");
    // admission by device memory: the configured budget and what is free now
    const size_t need = session_bytes_estimate(params->n + 1, space->kind);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        const size_t budget = sv->cfg.memory_budget ? (size_t)sv->cfg.memory_budget : free_b + sv->used_bytes;
        if (sv->used_bytes + need > budget || need + (size_t)(256u << 20) > free_b)
            return sfail(GMT_ERR_ADMISSION, "session refused: device memory budget exhausted");
        sv->used_bytes += need;
    }
    Session s;
    s.space = *space;
    s.goal = *goal;
    s.params = *params;
    std::memcpy(s.x_init, x_init, space->dim * sizeof(float));
    s.nbox = box_count;
    s.dp = space->pos_dim;
    s.bytes = need;
    const int P = s.dp;
    s.cur_lo.assign(box_lo, box_lo + box_count * P);
    s.cur_hi.assign(box_hi, box_hi + box_count * P);
    auto undo = [&](gmt_status st, const std::string& m) {
        if (s.graph) gmt_graph_free(s.graph);
        void* d[] = {s.d_lo, s.d_hi, s.aabb, s.verdict};
        for (void* p : d)
            if (p) cudaFree(p);
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->used_bytes -= need;
        return sfail(st, m);
    };
    cudaError_t e = cudaMalloc(&s.d_lo, std::max(1, box_count * P) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s.d_hi, std::max(1, box_count * P) * sizeof(float));
    if (e == cudaSuccess && box_count)
        e = cudaMemcpyAsync(s.d_lo, box_lo, box_count * P * sizeof(float), cudaMemcpyHostToDevice, sv->setup);
    if (e == cudaSuccess && box_count)
        e = cudaMemcpyAsync(s.d_hi, box_hi, box_count * P * sizeof(float), cudaMemcpyHostToDevice, sv->setup);
    if (e != cudaSuccess) return undo(GMT_ERR_CUDA, std::string("session setup: ") + cudaGetErrorString(e));
    gmt_boxes bx{box_count, s.d_lo, s.d_hi};
    gmt_status st = gmt_build_graph(space, &bx, x_init, goal, params, &s.graph, sv->setup);
    if (st != GMT_OK) return undo(st, std::string("session graph: ") + gmt_last_error());
    gmt_graph_get_view(s.graph, &s.view);
    e = edge_cache_setup(s.view, *space, *params, &s.aabb, &s.verdict, sv->setup);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->setup);
    if (e != cudaSuccess) return undo(GMT_ERR_CUDA, std::string("session setup: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(sv->mu);
    s.id = sv->next_session++;
    *session = s.id;
    sv->sessions[s.id] = std::move(s);
    return GMT_OK;
}

gmt_status gmt_server_submit(gmt_server* sv, int32_t session, uint64_t request_id, const float* box_lo,
                             const float* box_hi, int32_t* parent, float* cost) {
    if (!sv) return sfail(GMT_ERR_INVALID, "server is NULL");
    Request rq;
    rq.id = request_id;
    rq.session = session;
    rq.parent = parent;
    rq.cost = cost;
    rq.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->sessions.find(session);
        if (it == sv->sessions.end() || it->second.closing) return sfail(GMT_ERR_INVALID, "no such session");
        const int n = it->second.nbox * it->second.dp;
        if (n > 0 && (!box_lo || !box_hi)) return sfail(GMT_ERR_INVALID, "box arrays are NULL");
        rq.lo.assign(box_lo, box_lo + n);
        rq.hi.assign(box_hi, box_hi + n);
        sv->queue.push_back(std::move(rq));
    }
    sv->cv.notify_all();
    return GMT_OK;
}

gmt_status gmt_server_poll(gmt_server* sv, gmt_server_result* out, int32_t max, int32_t* count, int32_t wait_ms) {
    if (!sv || !out || !count || max < 1) return sfail(GMT_ERR_INVALID, "bad poll arguments");
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->done.empty() && wait_ms > 0)
        sv->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !sv->done.empty(); });
    const int n = std::min<int>(max, (int)sv->done.size());
    std::copy(sv->done.begin(), sv->done.begin() + n, out);
    sv->done.erase(sv->done.begin(), sv->done.begin() + n);
    *count = n;
    return GMT_OK;
}

gmt_status gmt_server_close_session(gmt_server* sv, int32_t session) {
    if (!sv) return sfail(GMT_ERR_INVALID, "server is NULL");
    Session s;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->sessions.find(session);
        if (it == sv->sessions.end()) return sfail(GMT_ERR_INVALID, "no such session");
        it->second.closing = true;
        // wait (bounded) until its queued and running requests are done
        const bool idle = sv->cv.wait_for(lk, std::chrono::seconds(30), [&] {
            bool queued = false;
            for (auto& q : sv->queue) queued = queued || q.session == session;
            return !queued && !sv->sessions[session].busy && !sv->sessions[session].moving;
        });
        if (!idle) {
            sv->sessions[session].closing = false;
            return sfail(GMT_ERR_TIMEOUT, "session still busy after 30 s");
        }
        s = std::move(sv->sessions[session]);
        sv->sessions.erase(session);
        sv->used_bytes -= s.bytes;
    }
    gmt_graph_free(s.graph);
    void* d[] = {s.d_lo, s.d_hi, s.aabb, s.verdict};
    for (void* p : d)
        if (p) cudaFree(p);
    return GMT_OK;
}

gmt_status gmt_server_move_start(gmt_server* sv, int32_t session, const float* x_init) {
    if (!sv || !x_init) return sfail(GMT_ERR_INVALID, "server and x_init must be non-NULL");
    gmt_space space;
    gmt_goal goal;
    gmt_params params;
    std::vector<float> lo, hi;
    gmt_boxes bx;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->sessions.find(session);
        if (it == sv->sessions.end() || it->second.closing) return sfail(GMT_ERR_INVALID, "no such session");
        if (it->second.moving) return sfail(GMT_ERR_INVALID, "the session's start is already being moved");
        // wait (bounded) until the requests submitted before the move are done
        const bool idle = sv->cv.wait_for(lk, std::chrono::seconds(30), [&] {
            bool queued = false;
            for (auto& q : sv->queue) queued = queued || q.session == session;
            auto s = sv->sessions.find(session);
            return s == sv->sessions.end() || (!queued && !s->second.busy);
        });
        it = sv->sessions.find(session);
        if (it == sv->sessions.end()) return sfail(GMT_ERR_INVALID, "the session was closed");
        if (!idle) return sfail(GMT_ERR_TIMEOUT, "session still busy after 30 s");
        Session& s = it->second;
        s.moving = true;  // requests submitted from now on wait for the new graph
        space = s.space; goal = s.goal; params = s.params;
        lo = s.cur_lo; hi = s.cur_hi;
        bx = gmt_boxes{s.nbox, s.d_lo, s.d_hi};
    }
    auto finish = [&](gmt_status st, const std::string& m) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            auto it = sv->sessions.find(session);
            if (it != sv->sessions.end()) it->second.moving = false;
        }
        sv->cv.notify_all();
        return st == GMT_OK ? GMT_OK : sfail(st, m);
    };
    // the new start must lie in X and outside the boxes the session has now
    for (int a = 0; a < space.dim; ++a)
        if (!(space.lo[a] <= x_init[a] && x_init[a] <= space.hi[a]))
            return finish(GMT_ERR_INVALID, "the new start is outside the state bounds");
    const int P = space.pos_dim;
    for (int b = 0; b < bx.count; ++b) {
        bool in = true;
        for (int a = 0; a < P; ++a) in = in && lo[(size_t)b * P + a] <= x_init[a] && x_init[a] <= hi[(size_t)b * P + a];
        if (in) return finish(GMT_ERR_INVALID, "the new start is inside a box");
    }
    // a new graph (same seed, the current boxes) in a handle of its own, so a
    // failure leaves the session as it was
    gmt_graph* ng = nullptr;
    gmt_status st = gmt_build_graph(&space, &bx, x_init, &goal, &params, &ng, sv->setup);
    if (st != GMT_OK) {
        const std::string m = std::string("start move: ") + gmt_last_error();
        if (ng) gmt_graph_free(ng);
        return finish(st, m);
    }
    gmt_graph_view nv;
    gmt_graph_get_view(ng, &nv);
    float* naabb = nullptr;
    uint8_t* nverdict = nullptr;
    cudaError_t e = edge_cache_setup(nv, space, params, &naabb, &nverdict, sv->setup);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->setup);
    if (e != cudaSuccess) {
        gmt_graph_free(ng);
        if (naabb) cudaFree(naabb);
        if (nverdict) cudaFree(nverdict);
        return finish(GMT_ERR_CUDA, std::string("start move: ") + cudaGetErrorString(e));
    }
    gmt_graph* og = nullptr;
    float* oaabb = nullptr;
    uint8_t* overdict = nullptr;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->sessions.find(session);
        if (it == sv->sessions.end()) {  // closing waits for the move, so this does not happen
            gmt_graph_free(ng);
            cudaFree(naabb);
            cudaFree(nverdict);
            return sfail(GMT_ERR_INVALID, "the session was closed");
        }
        Session& s = it->second;
        og = s.graph; oaabb = s.aabb; overdict = s.verdict;
        s.graph = ng; s.view = nv; s.aabb = naabb; s.verdict = nverdict;
        std::memcpy(s.x_init, x_init, space.dim * sizeof(float));
    }
    gmt_graph_free(og);
    cudaFree(oaabb);
    cudaFree(overdict);
    return finish(GMT_OK, "");
}

gmt_status gmt_server_session_view(gmt_server* sv, int32_t session, gmt_graph_view* view) {
    if (!sv || !view) return sfail(GMT_ERR_INVALID, "bad arguments");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->sessions.find(session);
    if (it == sv->sessions.end()) return sfail(GMT_ERR_INVALID, "no such session");
    *view = it->second.view;
    return GMT_OK;
}

}  // extern "C"
