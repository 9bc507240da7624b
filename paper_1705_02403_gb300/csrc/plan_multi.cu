// Lockstep batched wavefront: every query of a batch advances by one
// iteration of Algorithm 1 per super-iteration of one persistent cooperative
// grid, so the whole GPU works on the union of all queries' groups,
// candidates and checks instead of one team per query.
//
// The open lists, group lists and the candidate work of all queries are flat
// and shared: an open entry is (node, cost bits, query), a group entry
// (query, node).  Each block keeps a replicated table of the per-query
// iteration state (threshold index i, theta_i, live flag) in shared memory and
// updates it identically after every super-iteration from the per-query
// counters, so no block waits for another to publish it.
//
// One super-iteration, separated by two bounded grid barriers:
//
//   A  snapshot update of the previous iteration (closed group -> +inf, new
//      open nodes -> their cost) and group selection: every open entry of a
//      live query is split into G_i (cost <= theta_i of its query) and the
//      entries that stay open (keep segment of the next open list).
//   B+C per block: one warp per group entry pushes its out-row (one atomicMax
//      per neighbour claims it for this iteration), claimed candidates go to
//      the block's shared-memory queue, then the block's warps take the lazy
//      parent of each queued candidate over the iteration's open snapshot,
//      check that one edge and commit.  Push and pull need no barrier between
//      them: the snapshot is not written in this phase, and the claim is made
//      once per node and iteration whatever the order.  New open nodes fill
//      the next open list from its end (new segment), so keep and new entries
//      never share a counter.
//
// Per-query sums of a step (open count, minimum open cost, goal flag, edge
// counters) are first gathered per block in shared memory and reach the
// per-query control blocks once per block and step; list appends are
// reserved once per block (groups and kept entries with one packed 64-bit
// atomic).  Then every block evaluates the termination test and the next threshold for every live
// query: success, failure, or the next threshold index with the skip-ahead
// over empty groups.
// Results equal those of the single-query kernel bit for bit (the wavefront's
// outcome does not depend on the order of work within an iteration).
#include "plan_core.cuh"

namespace gmtk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Shared memory of one block: the replicated per-query state, the per-query
// sums of the current step, the candidate queue and the staged commits.
struct LockSmem {
    int4 commit[kLockQueue];          // (node, cost bits, query, 0) of the queue's commits
    int2 queue[kLockQueue];           // (query, node) candidates claimed by this block
    long long idx[kLockMaxQueries];   // threshold index i of every query
    unsigned long long app, app_base; // packed (groups, kept) block appends
    float theta[kLockMaxQueries];
    int live[kLockMaxQueries], status[kLockMaxQueries], iters[kLockMaxQueries];
    int base[kLockMaxQueries + 1];
    // sums of this step, flushed to the queries' PlanCtl at its end
    unsigned acc_min[kLockMaxQueries];
    int acc_open[kLockMaxQueries], acc_goal[kLockMaxQueries];
    unsigned acc_push[kLockMaxQueries], acc_pull[kLockMaxQueries], acc_checks[kLockMaxQueries];
    unsigned acc_failed[kLockMaxQueries], acc_computed[kLockMaxQueries];
    int nqueue, ncommit, commit_base;
};

__device__ __forceinline__ int find_node_query(const int* base, int nq, int g) {
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Lazy parent, check and commit for one candidate x of query q, run by a whole warp: lazy parent
// over the open snapshot, one edge check, commit.  Returns (uniformly across
// the warp) whether x joined the tree; its cost is then in *out_cost.
template <int KIND, int DP>
__device__ bool pull_candidate(const PlanArgs* __restrict__ Ap, LockSmem& sm, int q, const float* __restrict__ ocost,
                               int* stamp, int x, PlanCtl* team_ctl, float* out_cost) {
    constexpr int D = KIND == GMT_COST_DI ? 6 : (KIND == GMT_COST_DUBINS ? 4 : DP);
    const int lane = threadIdx.x & 31;
    const float INF = f_inf();
    const int* in_row = Ap->in_row;
    const int* in_col = Ap->in_col;
    const float* in_cost = Ap->in_cost;
    const float* X = Ap->X;
    const size_t pitch = (size_t)Ap->pitch;
    const int r0 = __ldg(&in_row[x]), r1 = __ldg(&in_row[x + 1]);
    float sx[D];
#pragma unroll
    for (int a = 0; a < D; ++a) sx[a] = __ldg(&X[(size_t)a * pitch + x]);
    float bc;
    int by, be;
    lane_parent_min<false>(in_col, in_cost, ocost, r0, r1, lane, &bc, &by, &be);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float oc = __shfl_xor_sync(kFull, bc, off);
        const int oy = __shfl_xor_sync(kFull, by, off);
        const int oe = __shfl_xor_sync(kFull, be, off);
        if (oc < bc || (oc == bc && oy < by)) { bc = oc; by = oy; be = oe; }
    }
    // The group node that pushed x is an open in-neighbour, so be >= 0; the
    // guard only keeps a broken invariant from reading out of bounds.
    if (be < 0) {
        if (lane == 0) {
            atomicAdd(&sm.acc_checks[q], 1u);
            atomicAdd(&sm.acc_failed[q], 1u);
            atomicCAS(&team_ctl->error, 0, (int)GMT_ERR_CUDA);
        }
        return false;
    }
    float sy[D];
#pragma unroll
    for (int a = 0; a < D; ++a) sy[a] = __ldg(&X[(size_t)a * pitch + by]);
    const int nbox = Ap->boxes.count;
    const float* blo = Ap->boxes.lo;
    const float* bhi = Ap->boxes.hi;
    uint8_t* verdict = Ap->verdict;
    bool free_edge;
    const int cached = verdict ? (int)__ldcg(&verdict[be]) : 0;
    if (cached != 0) {
        free_edge = cached == 1;
    } else {
        if (KIND == GMT_COST_EUCLID) {
            free_edge =
                segment_free_warp<DP>(sy, sx, __ldg(&in_cost[be]), Ap->seg_spacing, blo, bhi, nbox, Ap->grid);
        } else if (KIND == GMT_COST_DUBINS) {
            DubPath P;
            if (Ap->in_path) {
                const float4 w = __ldg(reinterpret_cast<const float4*>(Ap->in_path) + be);
                P = DubPath{__float_as_int(w.w), w.x, w.y, w.z, ((w.x + w.y) + w.z) * Ap->rho};
            } else {
                P = dubins_path(sy, sx, Ap->rho);
            }
            free_edge = dubins_free_warp(sy, sx, P, __ldg(&in_cost[be]), Ap->seg_spacing, Ap->rho, Ap->pos_lo,
                                         Ap->pos_hi, blo, bhi, nbox, Ap->grid);
        } else {
            const float tau = Ap->in_tau ? __ldg(&Ap->in_tau[be]) : di_tau(di_coef(sy, sx), Ap->r);
            free_edge = trajectory_free_warp(sy, sx, tau, Ap->traj_points, Ap->pos_lo, Ap->pos_hi, blo, bhi, nbox,
                                             Ap->grid);
        }
        if (lane == 0) {
            atomicAdd(&sm.acc_computed[q], 1u);
            if (verdict) verdict[be] = free_edge ? 1 : 2;
        }
    }
    if (lane == 0) {
        atomicAdd(&sm.acc_pull[q], (unsigned)(r1 - r0));
        atomicAdd(&sm.acc_checks[q], 1u);
        if (free_edge) {
            Ap->cost[x] = bc;
            Ap->parent[x] = by;
            stamp[x] = INT_MAX;
            atomicMin(&sm.acc_min[q], float_key(bc));
            atomicAdd(&sm.acc_open[q], 1);
        } else {
            atomicAdd(&sm.acc_failed[q], 1u);
        }
    }
    *out_cost = bc;
    return free_edge;
}

}  // namespace

template <int KIND, int DP>
__global__ void __launch_bounds__(1024) plan_lockstep_kernel(const PlanArgs* __restrict__ QA, int nq, LockScratch S,
                                                             GridTeam team) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LockSmem& sm = *reinterpret_cast<LockSmem*>(smem_raw);

    LockCtl* L = S.ctl;
    PlanCtl* tc = &L->team;
    const float INF = f_inf();
    const unsigned INF_KEY = 0x7f800000u;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, wpb = blockDim.x >> 5;
    const int rank = blockIdx.x * blockDim.x + tid, size = gridDim.x * blockDim.x;
    const int M = S.nodes;
    constexpr int kRunning = 1 << 30;

    for (int k = tid; k <= nq; k += blockDim.x) sm.base[k] = S.base[k];
    // per-query state; queries whose CSR did not fit their slice never start
    for (int k = tid; k < nq; k += blockDim.x) {
        const PlanArgs* A = &QA[k];
        int st = kRunning;
        if (A->check_edges) {
            const long long e = max(__ldcg(&A->out_row[A->N]), __ldcg(&A->in_row[A->N]));
            if (e > A->edge_cap) st = GMT_ERR_OOM;
        }
        if (st == kRunning && A->max_iters <= 0) st = GMT_ERR_ITER_LIMIT;
        sm.live[k] = st == kRunning;
        sm.status[k] = st;
        sm.iters[k] = 0;
        sm.idx[k] = 0;
        sm.theta[k] = 0.0f;
        sm.acc_min[k] = INF_KEY;
        sm.acc_open[k] = sm.acc_goal[k] = 0;
        sm.acc_push[k] = sm.acc_pull[k] = sm.acc_checks[k] = sm.acc_failed[k] = sm.acc_computed[k] = 0;
    }
    if (tid == 0) sm.app = 0;
    __syncthreads();

    // Initialisation for every query: x_init (node 0) is the only open node.
    for (int g = rank; g < M; g += size) {
        const int q = find_node_query(sm.base, nq, g);
        if (sm.status[q] == GMT_ERR_OOM) continue;
        const int v = g - sm.base[q];
        const float c0 = v == 0 ? 0.0f : INF;
        QA[q].cost[v] = c0;
        QA[q].parent[v] = -1;
        S.ocost[g] = c0;
        S.stamp[g] = v == 0 ? INT_MAX : -1;
    }
    for (int k = rank; k < nq; k += size) {
        PlanCtl* ctl = QA[k].ctl;
        ctl->min_keep[0] = ctl->min_keep[1] = INF_KEY;
        ctl->min_new[0] = ctl->min_new[1] = INF_KEY;
        ctl->goal_key = ~0ull;
        if (sm.live[k]) {
            // kept entries of open list 0 are counted in the high half of gk[1]
            const unsigned long long slot = atomicAdd(&L->gk[1], 1ull << 32) >> 32;
            S.open[0][slot] = make_int4(0, __float_as_int(0.0f), k, 0);
        }
    }
    int any = 0;
    for (int k = tid; k < nq; k += blockDim.x) any |= sm.live[k];
    any = __syncthreads_or(any);
    bool ok = team.sync(tc);

    // p: parity of this step's group list and open list (the next open list is p ^ 1)
    int it = 0, p = 0;
    while (ok && any) {
        const int4* cur = S.open[p];
        int4* nxt = S.open[p ^ 1];
        int2* G = S.glist[p];
        const unsigned long long gk_prev = __ldcg(&L->gk[p ^ 1]);
        const int nk = (int)(gk_prev >> 32), nn = ldcg_i(&L->new_total[p]);

        // ---- phase A: snapshot update of the previous step, group selection
        if (it > 0) {
            const int ngp = (int)(gk_prev & 0xffffffffu);
            const int2* Gp = S.glist[p ^ 1];
            for (int t = rank; t < ngp; t += size) {
                const int2 e = __ldcg(&Gp[t]);
                S.ocost[sm.base[e.x] + e.y] = INF;
            }
            for (int t = rank; t < nn; t += size) {
                const int4 e = __ldcg(&cur[M - 1 - t]);
                S.ocost[sm.base[e.z] + e.x] = __int_as_float(e.y);
            }
        }
        {
            const int ncur = nk + nn;
            for (int base = blockIdx.x * blockDim.x; base < ncur; base += size) {  // uniform per block
                const int t = base + tid;
                bool in_g = false, keep = false;
                int4 e = make_int4(0, 0, 0, 0);
                if (t < ncur) {
                    e = __ldcg(&cur[t < nk ? t : M - 1 - (t - nk)]);
                    if (sm.live[e.z]) {
                        in_g = __int_as_float(e.y) <= sm.theta[e.z];
                        keep = !in_g;
                    }
                }
                const unsigned mg = __ballot_sync(kFull, in_g), mk = __ballot_sync(kFull, keep);
                unsigned long long woff = 0;
                if (lane == 0 && (mg | mk))
                    woff = atomicAdd(&sm.app, ((unsigned long long)__popc(mk) << 32) | __popc(mg));
                woff = __shfl_sync(kFull, woff, 0);
                __syncthreads();
                if (tid == 0) {
                    const unsigned long long tot = sm.app;
                    sm.app_base = tot ? atomicAdd(&L->gk[p], tot) : 0ull;
                    sm.app = 0;
                }
                __syncthreads();
                const unsigned long long bb = sm.app_base;
                const unsigned below = (1u << lane) - 1u;
                if (in_g) {
                    const int sg = (int)(bb & 0xffffffffu) + (int)(woff & 0xffffffffu) + __popc(mg & below);
                    G[sg] = make_int2(e.z, e.x);
                    if (QA[e.z].is_goal[e.x]) sm.acc_goal[e.z] = 1;
                }
                if (keep) {
                    const int sk = (int)(bb >> 32) + (int)(woff >> 32) + __popc(mk & below);
                    nxt[sk] = e;
                    atomicMin(&sm.acc_min[e.z], float_key(__int_as_float(e.y)));
                    atomicAdd(&sm.acc_open[e.z], 1);
                }
            }
        }
        if (!(ok = team.sync(tc))) break;

        // ---- phase B+C: push from the groups, pull the block's candidates
        if (rank == 0) {
            L->gk[p ^ 1] = 0ull;   // previous group list and the kept count of this step's list: consumed
            L->new_total[p] = 0;
        }
        for (int k = rank; k < nq; k += size) {
            PlanCtl* ctl = QA[k].ctl;
            ctl->min_keep[p ^ 1] = INF_KEY;
            ctl->goal_flag[p ^ 1] = 0;
            ctl->open_count[p] = 0;
        }
        if (tid == 0) {
            sm.nqueue = 0;
            sm.ncommit = 0;
        }
        __syncthreads();
        {
            const int ng = (int)(__ldcg(&L->gk[p]) & 0xffffffffu);
            const int nwarps = gridDim.x * wpb;
            // group entries dealt round-robin over blocks first, then warps
            for (int gi = wib * gridDim.x + blockIdx.x; gi < ng; gi += nwarps) {
                const int2 ge = __ldcg(&G[gi]);
                const int q = ge.x, z = ge.y;
                const PlanArgs* A = &QA[q];
                const int* out_col = A->out_col;
                int* stamp = S.stamp + sm.base[q];
                const int e0 = __ldg(&A->out_row[z]), e1 = __ldg(&A->out_row[z + 1]);
                if (lane == 0) atomicAdd(&sm.acc_push[q], (unsigned)(e1 - e0));
                for (int eb = e0; eb < e1; eb += 32) {
                    const int e = eb + lane;
                    bool want = false;
                    int x = -1;
                    if (e < e1) {
                        x = __ldg(&out_col[e]);
                        want = atomicMax(&stamp[x], it) < it;
                    }
                    const unsigned wm = __ballot_sync(kFull, want);
                    if (!wm) continue;
                    int slot0 = 0;
                    if (lane == 0) slot0 = atomicAdd(&sm.nqueue, __popc(wm));
                    slot0 = __shfl_sync(kFull, slot0, 0);
                    const int my = slot0 + __popc(wm & ((1u << lane) - 1u));
                    if (want && my < kLockQueue) sm.queue[my] = make_int2(q, x);
                    // claims that do not fit the queue are pulled by this warp now
                    unsigned over = __ballot_sync(kFull, want && my >= kLockQueue);
                    while (over) {
                        const int src = __ffs(over) - 1;
                        over &= over - 1;
                        const int xo = __shfl_sync(kFull, x, src);
                        float c;
                        if (pull_candidate<KIND, DP>(A, sm, q, S.ocost + sm.base[q], stamp, xo, tc, &c) &&
                            lane == 0) {
                            const int s = atomicAdd(&L->new_total[p ^ 1], 1);
                            nxt[M - 1 - s] = make_int4(xo, __float_as_int(c), q, 0);
                        }
                    }
                }
            }
        }
        __syncthreads();
        {
            const int nqueue = min(sm.nqueue, kLockQueue);
            for (int t = wib; t < nqueue; t += wpb) {
                const int2 c = sm.queue[t];
                float cost;
                if (pull_candidate<KIND, DP>(&QA[c.x], sm, c.x, S.ocost + sm.base[c.x], S.stamp + sm.base[c.x], c.y, tc,
                                             &cost) &&
                    lane == 0) {
                    const int s = atomicAdd(&sm.ncommit, 1);
                    sm.commit[s] = make_int4(c.y, __float_as_int(cost), c.x, 0);
                }
            }
        }
        __syncthreads();
        {
            const int nc = sm.ncommit;
            if (tid == 0 && nc > 0) sm.commit_base = atomicAdd(&L->new_total[p ^ 1], nc);
            // the step's per-query sums of this block
            for (int k = tid; k < nq; k += blockDim.x) {
                const int n_open = sm.acc_open[k];
                if (n_open == 0 && sm.acc_goal[k] == 0 && sm.acc_push[k] == 0 && sm.acc_checks[k] == 0) continue;
                PlanCtl* ctl = QA[k].ctl;
                if (n_open) {
                    atomicAdd(&ctl->open_count[p ^ 1], n_open);
                    atomicMin(&ctl->min_keep[p], sm.acc_min[k]);
                }
                if (sm.acc_goal[k]) ctl->goal_flag[p] = 1;
                if (sm.acc_push[k]) atomicAdd(&ctl->push_edges, (unsigned long long)sm.acc_push[k]);
                if (sm.acc_checks[k]) {
                    atomicAdd(&ctl->pull_edges, (unsigned long long)sm.acc_pull[k]);
                    atomicAdd(&ctl->checks, (unsigned long long)sm.acc_checks[k]);
                    if (sm.acc_failed[k]) atomicAdd(&ctl->failed, (unsigned long long)sm.acc_failed[k]);
                    if (sm.acc_computed[k]) atomicAdd(&ctl->checks_computed, (unsigned long long)sm.acc_computed[k]);
                }
                sm.acc_min[k] = INF_KEY;
                sm.acc_open[k] = sm.acc_goal[k] = 0;
                sm.acc_push[k] = sm.acc_pull[k] = sm.acc_checks[k] = sm.acc_failed[k] = sm.acc_computed[k] = 0;
            }
            __syncthreads();
            for (int t = tid; t < nc; t += blockDim.x) nxt[M - 1 - (sm.commit_base + t)] = sm.commit[t];
        }
        if (!(ok = team.sync(tc))) break;

        // ---- termination test and next threshold for every live query (same result in every block)
        ++it;
        any = 0;
        for (int k = tid; k < nq; k += blockDim.x) {
            if (!sm.live[k]) continue;
            const PlanArgs* A = &QA[k];
            PlanCtl* ctl = A->ctl;
            const int goal = ldcg_i(&ctl->goal_flag[p]);
            const int n_open = ldcg_i(&ctl->open_count[p ^ 1]);
            const unsigned mk = ldcg_u(&ctl->min_keep[p]);
            int st = kRunning;
            if (goal) {
                st = GMT_OK;
            } else if (n_open == 0) {
                st = GMT_NO_PATH;
            } else {
                const float m = __uint_as_float(mk);
                const float delta = A->delta;
                const long long i = sm.idx[k];
                if (delta == 0.0f) {
                    sm.theta[k] = m;
                    sm.idx[k] = i + 1;
                } else {
                    const float qk = m / delta;
                    if (!(qk < 16777216.0f)) {
                        st = GMT_ERR_ITER_LIMIT;  // i stays below 2^24
                    } else {
                        long long kk = (long long)ceilf(qk);
                        if (kk < i + 1) kk = i + 1;
                        while (kk > i + 1 && (float)(kk - 1) * delta >= m) --kk;
                        while ((float)kk * delta < m) ++kk;
                        sm.idx[k] = kk;
                        sm.theta[k] = (float)kk * delta;
                    }
                }
                if (st == kRunning && it >= A->max_iters) st = GMT_ERR_ITER_LIMIT;
            }
            if (st != kRunning) {
                sm.live[k] = 0;
                sm.status[k] = st;
                sm.iters[k] = it;
            } else {
                any = 1;
            }
        }
        any = __syncthreads_or(any);
        p ^= 1;
    }

    // ---- result: tree sizes and minimum-cost goal nodes (ties by index)
    if (ok) {
        const int gwarp = rank >> 5, nwarps = size >> 5;
        for (int base = gwarp * 32; base < M; base += nwarps * 32) {
            const int g = base + lane;
            int q = -1;
            bool in_tree = false;
            if (g < M) {
                q = find_node_query(sm.base, nq, g);
                if (sm.status[q] != GMT_ERR_OOM) {
                    const PlanArgs* A = &QA[q];
                    const int v = g - sm.base[q];
                    const float c = ldcg_f(&A->cost[v]);
                    in_tree = c < INF;
                    if (in_tree && sm.status[q] == GMT_OK && A->is_goal[v])
                        atomicMin(&A->ctl->goal_key, ((unsigned long long)float_key(c) << 32) | (unsigned)v);
                }
            }
            unsigned todo = __ballot_sync(kFull, in_tree);
            while (todo) {
                const int leader = __ffs(todo) - 1;
                const int qk = __shfl_sync(kFull, q, leader);
                const unsigned grp = __ballot_sync(kFull, in_tree && q == qk);
                if (lane == leader) atomicAdd(&QA[qk].ctl->tree_size, (unsigned long long)__popc(grp));
                todo &= ~grp;
            }
        }
        ok = team.sync(tc);
    }
    // ---- per query: status, iteration counts, goal node and path
    for (int k = rank; k < nq; k += size) {
        const PlanArgs* A = &QA[k];
        PlanCtl* ctl = A->ctl;
        if (sm.status[k] == GMT_ERR_OOM) {
            ctl->status = GMT_ERR_OOM;
            ctl->goal_node = -1;
            continue;
        }
        const int err = ld_volatile(&tc->error);
        ctl->status = err ? err : sm.status[k];
        ctl->iters = sm.iters[k];
        ctl->final_i = (int)sm.idx[k];
        ctl->goal_node = -1;
        ctl->path_len = 0;
        if (ok && !err && sm.status[k] == GMT_OK) {
            const int N = A->N;
            const int g = (int)(__ldcg(&ctl->goal_key) & 0xffffffffu);
            ctl->goal_node = g;
            int len = 1, v = g;
            while (v > 0 && len <= N) {
                v = ldcg_i(&A->parent[v]);
                ++len;
            }
            if (v != 0) len = 0;  // not a chain back to x_init: report no path
            ctl->path_len = len;
            if (A->path) {
                v = g;
                for (int j = len - 1; j >= 0; --j) {
                    A->path[j] = v;
                    if (v > 0) v = ldcg_i(&A->parent[v]);
                }
            }
        }
    }
}

// ----------------------------------------------------------------- launcher
namespace {
template <int KIND, int DP>
cudaError_t lockstep_t(const PlanArgs* queries, int nq, const LockScratch& s, int blocks, int threads,
                       cudaStream_t st) {
    auto kern = plan_lockstep_kernel<KIND, DP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LockSmem));
    if (e != cudaSuccess) return e;
    GridTeam team;
    team.expected = (unsigned)blocks;
    team.spin_limit = kDefaultSpinLimit;
    LockScratch sc = s;
    const PlanArgs* q = queries;
    int n = nq;
    void* params[] = {(void*)&q, &n, &sc, &team};
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(threads), params, sizeof(LockSmem), st);
}

template <int KIND, int DP>
int lockstep_blocks_t(int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto kern = plan_lockstep_kernel<KIND, DP>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LockSmem)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sizeof(LockSmem)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}
}  // namespace

cudaError_t launch_plan_lockstep(int kind, int dp, const PlanArgs* queries, int nq, const LockScratch& s, int blocks,
                                 int threads, cudaStream_t st) {
    if (nq < 1 || nq > kLockMaxQueries || blocks < 1) return cudaErrorInvalidValue;
    if (kind == GMT_COST_DI) return lockstep_t<GMT_COST_DI, 3>(queries, nq, s, blocks, threads, st);
    if (kind == GMT_COST_DUBINS) return lockstep_t<GMT_COST_DUBINS, 3>(queries, nq, s, blocks, threads, st);
    if (dp == 2) return lockstep_t<GMT_COST_EUCLID, 2>(queries, nq, s, blocks, threads, st);
    if (dp == 3) return lockstep_t<GMT_COST_EUCLID, 3>(queries, nq, s, blocks, threads, st);
    return cudaErrorInvalidValue;
}

int plan_lockstep_max_blocks(int kind, int dp, int threads) {
    if (kind == GMT_COST_DI) return lockstep_blocks_t<GMT_COST_DI, 3>(threads);
    if (kind == GMT_COST_DUBINS) return lockstep_blocks_t<GMT_COST_DUBINS, 3>(threads);
    if (dp == 2) return lockstep_blocks_t<GMT_COST_EUCLID, 2>(threads);
    if (dp == 3) return lockstep_blocks_t<GMT_COST_EUCLID, 3>(threads);
    return 0;
}

}  // namespace gmtk
