// Batched wavefront as one pool of work items (the pool scheme of
// gmt_plan_batch): every warp of one persistent launch takes work from any
// query, so queries of every kind and size advance together and no query waits
// at a team barrier for the slowest member of its team.
//
// Each iteration of Algorithm 1 on one query runs as three stages of work
// items, each stage's item count fixed when it is published:
//   SELECT  32 entries of the open list: group selection (cost <= theta_i),
//           kept entries to the next open list, group nodes to the group list;
//   PUSH    two nodes z of the group: their out-rows are scanned and every
//           unexplored neighbour is claimed once per iteration (its stamp is
//           read first, so only unclaimed ones cost an atomic) and appended to
//           the candidate list;
//   PULL    two candidates x: lazy parent over the in-row against the open-set
//           snapshot, one collision check, commit.
// A warp claims an item with one atomic add on the query's claim word, which
// also returns the stage and its item count (claims past the count are
// ignored); the warp that completes a stage's last item publishes the next
// stage, and after PULL runs the termination test, computes the next
// threshold and publishes the next iteration's SELECT stage.  Nothing ever
// waits for another warp, so no barrier holds warps idle and every query
// advances at its own pace.
//
// The open-set snapshot is double-buffered: iteration i reads buffer i & 1
// (open as of the start of the iteration, Sec. III-A's V_open) and writes the
// snapshot of iteration i + 1 into the other buffer, which still holds that
// of iteration i - 1: the previous group closes, the nodes opened in i - 1
// open (unless they join G_i), G_i closes, and every commit of iteration i
// opens its node.  No separate snapshot update is needed between iterations.
//
// Every wait is bounded: a worker that finds no work for kPoolIdleLimit
// rounds records GMT_ERR_TIMEOUT and the kernel ends; queries that did not
// finish keep the status GMT_ERR_TIMEOUT set at their start.  The caller
// zeroes the PoolCtl block before the launch.  Progress never depends on
// another warp being resident: a claimed item is always completed without
// waiting for other items.
#include "plan_core.cuh"

namespace gmtk {

namespace {

constexpr int kPoolSel = 32;        // open-list entries per SELECT item
constexpr int kPoolPush = 2;        // group nodes per PUSH item
constexpr int kPoolPull = 2;        // candidates per PULL item
constexpr int kPoolHomePolls = 16;  // polls of an idle home query before helping another
constexpr int kPoolIdleLimit = 1 << 22;

// Claim word: bits 0-23 items claimed, 24-47 items of the stage, 48-49 stage.
enum { kStageSelect = 0, kStagePush = 1, kStagePull = 2, kStageNone = 3 };
__host__ __device__ constexpr unsigned long long stage_word(int stage, int items) {
    return ((unsigned long long)stage << 48) | ((unsigned long long)items << 24);
}
__device__ __forceinline__ int word_stage(unsigned long long w) { return (int)(w >> 48) & 3; }
__device__ __forceinline__ int word_items(unsigned long long w) { return (int)(w >> 24) & 0xffffff; }
__device__ __forceinline__ int word_claimed(unsigned long long w) { return (int)(w & 0xffffff); }
__device__ __forceinline__ bool has_work(unsigned long long w) {
    return word_stage(w) != kStageNone && word_claimed(w) < word_items(w);
}

__device__ __forceinline__ unsigned long long ldcg_u64(const unsigned long long* p) { return __ldcg(p); }

// Atomics with the ordering the protocol needs (GPU scope).
__device__ __forceinline__ unsigned long long add_acquire(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acquire.gpu.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ int add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void exch_release(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.release.gpu.exch.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    (void)old;
}

// Lane 0: one item of the query's current stage, if it has one unclaimed.
// Returns the stage (-1: nothing claimed), the item index and the stage's
// item count.
__device__ __forceinline__ int pool_claim(PoolQ& Q, int* item, int* items) {
    if (!has_work(ldcg_u64(&Q.word))) return -1;
    const unsigned long long old = add_acquire(&Q.word, 1ull);
    if (!has_work(old)) return -1;
    *item = word_claimed(old);
    *items = word_items(old);
    return word_stage(old);
}

struct TaskCounters {
    unsigned long long push = 0, pull = 0;
    unsigned checks = 0, failed = 0, computed = 0, tree = 0;
};

__device__ __forceinline__ void flush_counters(PlanCtl* ctl, const TaskCounters& c) {
    if (c.push) atomicAdd(&ctl->push_edges, c.push);
    if (c.pull) atomicAdd(&ctl->pull_edges, c.pull);
    if (c.checks) atomicAdd(&ctl->checks, (unsigned long long)c.checks);
    if (c.failed) atomicAdd(&ctl->failed, (unsigned long long)c.failed);
    if (c.computed) atomicAdd(&ctl->checks_computed, (unsigned long long)c.computed);
    if (c.tree) atomicAdd(&ctl->tree_size, (unsigned long long)c.tree);
}

// ------------------------------------------------------------------ SELECT
// Entries t = 32 j + lane of the open list (kept entries at its front, the
// nodes opened by the previous iteration at its back) and of the previous
// group list.
__device__ void select_item(const PlanArgs& A, int j, const PoolIter& I) {
    const int lane = threadIdx.x & 31;
    const int N = A.N, p = I.it & 1;
    const float INF = f_inf();
    const unsigned INF_KEY = 0x7f800000u;
    PlanCtl* ctl = A.ctl;
    const int2* cur = A.list_open[p];
    int2* nxt = A.list_open[p ^ 1];
    int* G = A.list_g[p];
    int* Gprev = A.list_g[p ^ 1];
    float* onext = A.ocost + (size_t)(p ^ 1) * N;
    const int t = j * kPoolSel + lane;
    // the previous group closed: not open from this iteration on
    if (t < I.ng_prev) onext[__ldcg(&Gprev[t])] = INF;
    bool in_g = false, keep = false;
    int2 e = make_int2(-1, 0);
    if (t < I.ncur) {
        e = __ldcg(&cur[t < I.nk ? t : N - 1 - (t - I.nk)]);
        in_g = __int_as_float(e.y) <= I.theta;
        keep = !in_g;
        if (in_g) onext[e.x] = INF;                               // G_i closes
        else if (t >= I.nk) onext[e.x] = __int_as_float(e.y);     // opened in i - 1, stays open
        if (in_g && A.is_goal[e.x]) ctl->goal_flag[p] = 1;
    }
    const unsigned mg = __ballot_sync(0xffffffffu, in_g), mkeep = __ballot_sync(0xffffffffu, keep);
    const unsigned below = (1u << lane) - 1u;
    if (mkeep | mg) {
        // one atomic reserves the warp's group entries and kept entries
        unsigned long long base = 0;
        if (lane == 0)
            base = atomicAdd(&ctl->gk[p], ((unsigned long long)__popc(mkeep) << 32) | __popc(mg));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) nxt[(int)(base >> 32) + __popc(mkeep & below)] = e;
        if (in_g) G[(int)(base & 0xffffffffu) + __popc(mg & below)] = e.x;
        const unsigned kmin = __reduce_min_sync(0xffffffffu, keep ? float_key(__int_as_float(e.y)) : INF_KEY);
        if (lane == 0 && kmin != INF_KEY) atomicMin(&ctl->min_keep[p], kmin);
    }
}

// -------------------------------------------------------------------- PUSH
// Group nodes G[j kPoolPush ..] (at most kPoolPush): every unexplored
// out-neighbour is claimed for this iteration (stamp: INT_MAX once in the
// tree, else the last iteration that claimed it) and appended to the
// candidate list.
__device__ void push_item(const PlanArgs& A, int j, const PoolIter& I, TaskCounters& cnt) {
    const int lane = threadIdx.x & 31;
    const int p = I.it & 1, it = I.it;
    PlanCtl* ctl = A.ctl;
    const int* G = A.list_g[p];
    const int g1 = min((j + 1) * kPoolPush, I.ng);
    for (int g = j * kPoolPush; g < g1; ++g) {
        const int z = __ldcg(&G[g]);
        const int e0 = __ldg(&A.out_row[z]), e1 = __ldg(&A.out_row[z + 1]);
        if (lane == 0) cnt.push += (unsigned long long)(e1 - e0);
        for (int eb = e0; eb < e1; eb += 4 * 32) {
            int xs[4];
            bool want[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int ei = eb + 32 * c + lane;
                xs[c] = ei < e1 ? __ldg(&A.out_col[ei]) : -1;
            }
            int st[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) st[c] = xs[c] >= 0 ? __ldcg(&A.stamp[xs[c]]) : INT_MAX;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                // stamps only grow, so a stamp already >= it (in the tree, or
                // claimed this iteration) is final; otherwise one atomic both
                // tests and claims
                want[c] = st[c] < it && atomicMax(&A.stamp[xs[c]], it) < it;
            unsigned m[4];
            int total = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                m[c] = __ballot_sync(0xffffffffu, want[c]);
                total += __popc(m[c]);
            }
            if (total == 0) continue;
            int slot = 0;
            if (lane == 0) slot = atomicAdd(&ctl->cand_count[p], total);
            slot = __shfl_sync(0xffffffffu, slot, 0);
            const unsigned below = (1u << lane) - 1u;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (want[c]) A.list_cand[slot + __popc(m[c] & below)] = xs[c];
                slot += __popc(m[c]);
            }
        }
    }
}

// -------------------------------------------------------------------- PULL
// Candidates list_cand[j kPoolPull ..] (at most kPoolPull): lazy parent (minimum (cost, index)
// over the in-neighbours open in the snapshot), one collision check, commit.
template <int KIND, int DP>
__device__ void pull_item(const PlanArgs& A, int j, const PoolIter& I, TaskCounters& cnt) {
    constexpr int D = KIND == GMT_COST_DI ? 6 : (KIND == GMT_COST_DUBINS ? 4 : DP);
    const int lane = threadIdx.x & 31;
    const int N = A.N, p = I.it & 1;
    PlanCtl* ctl = A.ctl;
    const float* ocur = A.ocost + (size_t)p * N;
    float* onext = A.ocost + (size_t)(p ^ 1) * N;
    int2* nxt = A.list_open[p ^ 1];
    const int c1 = min((j + 1) * kPoolPull, I.nc);
    for (int ci = j * kPoolPull; ci < c1; ++ci) {
        const int x = __ldcg(&A.list_cand[ci]);
        const int r0 = __ldg(&A.in_row[x]), r1 = __ldg(&A.in_row[x + 1]);
        const bool x_goal = A.is_goal[x] != 0;
        float sx[D];
#pragma unroll
        for (int a = 0; a < D; ++a) sx[a] = __ldg(&A.X[(size_t)a * A.pitch + x]);
        float bc;
        int by, be;
        lane_parent_min<false>(A.in_col, A.in_cost, ocur, r0, r1, lane, &bc, &by, &be);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float oc = __shfl_xor_sync(0xffffffffu, bc, off);
            const int oy = __shfl_xor_sync(0xffffffffu, by, off);
            const int oe = __shfl_xor_sync(0xffffffffu, be, off);
            if (oc < bc || (oc == bc && oy < by)) { bc = oc; by = oy; be = oe; }
        }
        // the group node that pushed x is an open in-neighbour, so be >= 0; the
        // guard keeps a broken invariant from reading out of bounds
        if (be < 0) {
            if (lane == 0) { ++cnt.checks; ++cnt.failed; atomicCAS(&ctl->error, 0, (int)GMT_ERR_CUDA); }
            continue;
        }
        if (lane == 0) cnt.pull += (unsigned long long)(r1 - r0);
        float sy[D];
#pragma unroll
        for (int a = 0; a < D; ++a) sy[a] = __ldg(&A.X[(size_t)a * A.pitch + by]);
        bool free_edge;
        const int cached = A.verdict ? (int)__ldcg(&A.verdict[be]) : 0;
        const float* blo = A.boxes.lo;
        const float* bhi = A.boxes.hi;
        if (cached != 0) {
            free_edge = cached == 1;
        } else {
            if (KIND == GMT_COST_EUCLID) {
                free_edge = segment_free_warp<DP>(sy, sx, __ldg(&A.in_cost[be]), A.seg_spacing, blo, bhi,
                                                  A.boxes.count, A.grid);
            } else if (KIND == GMT_COST_DUBINS) {
                DubPath P;
                if (A.in_path) {
                    const float4 w = __ldg(reinterpret_cast<const float4*>(A.in_path) + be);
                    P = DubPath{__float_as_int(w.w), w.x, w.y, w.z, ((w.x + w.y) + w.z) * A.rho};
                } else {
                    P = dubins_path(sy, sx, A.rho);
                }
                free_edge = dubins_free_warp(sy, sx, P, __ldg(&A.in_cost[be]), A.seg_spacing, A.rho, A.pos_lo,
                                             A.pos_hi, blo, bhi, A.boxes.count, A.grid);
            } else {
                const float tau = A.in_tau ? __ldg(&A.in_tau[be]) : di_tau(di_coef(sy, sx), A.r);
                free_edge = trajectory_free_warp(sy, sx, tau, A.traj_points, A.pos_lo, A.pos_hi, blo, bhi,
                                                 A.boxes.count, A.grid);
            }
            if (lane == 0) {
                ++cnt.computed;
                if (A.verdict) A.verdict[be] = free_edge ? 1 : 2;
            }
        }
        if (lane == 0) {
            ++cnt.checks;
            if (free_edge) {
                A.cost[x] = bc;
                A.parent[x] = by;
                A.stamp[x] = INT_MAX;
                onext[x] = bc;  // open from the next iteration on
                const int s = atomicAdd(&ctl->new_count[p ^ 1], 1);
                nxt[N - 1 - s] = make_int2(x, __float_as_int(bc));
                atomicMin(&ctl->min_new[p], float_key(bc));
                ++cnt.tree;
                if (x_goal) atomicMin(&ctl->goal_key, ((unsigned long long)float_key(bc) << 32) | (unsigned)x);
            } else {
                ++cnt.failed;
            }
        }
    }
}

template <int KIND, int DP>
__device__ __forceinline__ void run_item(const PlanArgs& A, int stage, int j, const PoolIter& I, TaskCounters& cnt) {
    if (stage == kStageSelect) select_item(A, j, I);
    else if (stage == kStagePush) push_item(A, j, I, cnt);
    else pull_item<KIND, DP>(A, j, I, cnt);
}

// ------------------------------------------------------------ iteration end
// Lane 0 of the warp that completed the iteration's last item: termination
// test (success if the group held a goal node, failure if nothing stays
// open), next threshold index (skipping indices whose group would be empty),
// then either the next iteration's SELECT items or the query's result.
__device__ void end_iteration(const PlanArgs& A, PoolQ& Q, const PoolIter& I, PoolCtl* pool) {
    PlanCtl* ctl = A.ctl;
    const int p = I.it & 1;
    const unsigned INF_KEY = 0x7f800000u;
    const int err = ld_volatile(&ctl->error);
    const int goal = __ldcg(&ctl->goal_flag[p]);
    const int kept = (int)(__ldcg(&ctl->gk[p]) >> 32);
    const int opened = __ldcg(&ctl->new_count[p ^ 1]);
    const int ngrp = (int)(__ldcg(&ctl->gk[p]) & 0xffffffffu);
    const unsigned mk = min(__ldcg(&ctl->min_keep[p]), __ldcg(&ctl->min_new[p]));
    const int it = I.it + 1;
    long long i = I.i;
    float theta = I.theta;
    constexpr int kRunning = 1 << 30;
    int status = kRunning;
    if (err) status = err;
    else if (goal) status = GMT_OK;
    else if (kept + opened == 0) status = GMT_NO_PATH;
    else {
        const float m = __uint_as_float(mk);
        if (A.delta == 0.0f) {
            theta = m;
            i = i + 1;
        } else {
            const float qk = m / A.delta;
            if (!(qk < 16777216.0f)) {
                status = GMT_ERR_ITER_LIMIT;  // the index stays below 2^24
            } else {
                long long k = (long long)ceilf(qk);
                if (k < i + 1) k = i + 1;
                while (k > i + 1 && (float)(k - 1) * A.delta >= m) --k;
                while ((float)k * A.delta < m) ++k;
                i = k;
                theta = (float)i * A.delta;
            }
        }
        if (status == kRunning && it >= A.max_iters) status = GMT_ERR_ITER_LIMIT;
    }
    if (status == kRunning) {
        // counters of the next iteration (parity p ^ 1); its commits count into new_count[p]
        const int q = p ^ 1;
        ctl->gk[q] = 0ull;
        ctl->cand_count[q] = 0;
        ctl->new_count[p] = 0;
        ctl->min_keep[q] = INF_KEY;
        ctl->min_new[q] = INF_KEY;
        ctl->goal_flag[q] = 0;
        PoolIter n;
        n.it = it;
        n.ncur = kept + opened;
        n.nk = kept;
        n.ng_prev = ngrp;
        n.theta = theta;
        n.i = i;
        n.ng = 0;
        n.nc = 0;
        Q.iter = n;
        Q.done = 0;
        exch_release(&Q.word, stage_word(kStageSelect, (max(n.ncur, n.ng_prev) + kPoolSel - 1) / kPoolSel));
        return;
    }
    // result: the goal node was tracked at each commit; the returned path is
    // walked back to x_init
    ctl->iters = it;
    ctl->final_i = (int)i;
    ctl->goal_node = -1;
    ctl->path_len = 0;
    if (status == GMT_OK) {
        const int g = (int)(__ldcg(&ctl->goal_key) & 0xffffffffu);
        ctl->goal_node = g;
        int len = 1, v = g;
        while (v > 0 && len <= A.N) {
            v = __ldcg(&A.parent[v]);
            ++len;
        }
        if (v != 0) len = 0;
        ctl->path_len = len;
        if (A.path) {
            v = g;
            for (int k = len - 1; k >= 0; --k) {
                A.path[k] = v;
                if (v > 0) v = __ldcg(&A.parent[v]);
            }
        }
    }
    ctl->status = status;
    atomicExch(&Q.word, stage_word(kStageNone, 0));
    __threadfence();
    atomicExch(&Q.live, 0);
    atomicAdd(&pool->finished, 1);
}

// Lane 0 of the warp that completed a stage's last item: the next stage
// (PUSH after SELECT, PULL after PUSH; an empty stage is skipped), or, after
// PULL, the end of the iteration.
__device__ void end_stage(const PlanArgs& A, PoolQ& Q, int stage, const PoolIter& I, PoolCtl* pool) {
    PlanCtl* ctl = A.ctl;
    const int p = I.it & 1;
    if (stage == kStageSelect) {
        const int ng = (int)(__ldcg(&ctl->gk[p]) & 0xffffffffu);
        if (ng > 0) {
            Q.iter.ng = ng;
            Q.done = 0;
            exch_release(&Q.word, stage_word(kStagePush, (ng + kPoolPush - 1) / kPoolPush));
            return;
        }
        stage = kStagePush;  // no group node: nothing to push
    }
    if (stage == kStagePush) {
        const int nc = __ldcg(&ctl->cand_count[p]);
        if (nc > 0) {
            Q.iter.nc = nc;
            Q.done = 0;
            exch_release(&Q.word, stage_word(kStagePull, (nc + kPoolPull - 1) / kPoolPull));
            return;
        }
    }
    end_iteration(A, Q, I, pool);
}

// One block per query: the wavefront's initial state (Alg. 1's
// initialisation: x_init is the only open node and the root of the tree).
__global__ void __launch_bounds__(256) pool_init_kernel(const PlanArgs* __restrict__ args,
                                                        const int* __restrict__ order, PoolQ* __restrict__ qs,
                                                        PoolCtl* pool) {
    const int pos = blockIdx.x;
    const PlanArgs& A = args[order[pos]];
    PoolQ& Q = qs[pos];
    const int N = A.N;
    const float INF = f_inf();
    const unsigned INF_KEY = 0x7f800000u;
    PlanCtl* ctl = A.ctl;
    bool oom = false;
    if (A.check_edges) oom = max(__ldcg(&A.out_row[N]), __ldcg(&A.in_row[N])) > A.edge_cap;
    if (!oom) {
        for (int v = threadIdx.x; v < N; v += blockDim.x) {
            const float c0 = v == 0 ? 0.0f : INF;
            A.cost[v] = c0;
            A.parent[v] = -1;
            A.stamp[v] = v == 0 ? INT_MAX : -1;
            A.ocost[v] = c0;
            A.ocost[(size_t)N + v] = c0;
        }
    }
    if (threadIdx.x == 0) {
        ctl->error = 0;
        ctl->iters = ctl->final_i = ctl->path_len = 0;
        ctl->goal_node = -1;
        ctl->push_edges = ctl->pull_edges = ctl->checks = ctl->failed = ctl->checks_computed = 0ull;
        ctl->tree_size = 1ull;
        for (int k = 0; k < 2; ++k) {
            ctl->gk[k] = 0ull;
            ctl->new_count[k] = ctl->cand_count[k] = 0;
            ctl->min_keep[k] = ctl->min_new[k] = INF_KEY;
            ctl->goal_flag[k] = 0;
        }
        ctl->goal_key = A.is_goal[0] ? 0ull : ~0ull;
        PoolIter n;
        n.it = 0; n.ncur = 1; n.nk = 1; n.ng_prev = 0; n.theta = 0.0f; n.i = 0; n.ng = 0; n.nc = 0;
        Q.iter = n;
        Q.done = 0;
        if (oom) {
            ctl->status = GMT_ERR_OOM;
            Q.word = stage_word(kStageNone, 0);
            Q.live = 0;
            atomicAdd(&pool->finished, 1);
        } else {
            A.list_open[0][0] = make_int2(0, __float_as_int(0.0f));
            // a query that has not finished when the kernel ends reports a timeout
            ctl->status = GMT_ERR_TIMEOUT;
            Q.live = 1;
            Q.word = stage_word(kStageSelect, 1);
        }
    }
}

// Kernel kinds: 0 double integrator, 1 Dubins airplane, 2 2D geometric, 3 3D geometric.
__device__ __forceinline__ int kernel_kind(const PlanArgs& A) {
    return A.kind == GMT_COST_DI ? 0 : A.kind == GMT_COST_DUBINS ? 1 : A.dp == 2 ? 2 : 3;
}

// Lane 0: the first query in order (largest first) with claimable work,
// spread over the first ones found by the warp index; claims on it.
__device__ __forceinline__ int scan_and_claim(PoolQ* qs, int nq, int wid, int* stage, int* item, int* items) {
    for (int base = 0; base < nq; base += 32) {
        unsigned m = 0;
        for (int l = 0; l < 32 && base + l < nq; ++l)
            if (has_work(ldcg_u64(&qs[base + l].word))) m |= 1u << l;
        if (!m) continue;
        int pick = wid % __popc(m);
        for (; pick > 0; --pick) m &= m - 1;
        const int pos = base + __ffs(m) - 1;
        *stage = pool_claim(qs[pos], item, items);
        return *stage >= 0 ? pos : -1;
    }
    return -1;
}

// Warps are dealt to queries in proportion to their edge counts (ecum: the
// running sum over the order, nq + 1 entries): a warp works on its home
// query while it has claimable items, helps the others (largest first) while
// its home waits for an iteration to end, and adopts another home once its
// own is done.
// ALL_KINDS = false: a lean instantiation for batches of geometric queries
// only (the double-integrator and Dubins checks need far more registers).
template <bool ALL_KINDS>
__global__ void __launch_bounds__(256) pool_kernel(const PlanArgs* __restrict__ args, const int* __restrict__ order,
                                                   const long long* __restrict__ ecum, int nq,
                                                   PoolQ* __restrict__ qs, PoolCtl* pool) {
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    // home: the query whose share of the edges holds this warp's position
    int home = 0;
    {
        const long long total = ecum[nq];
        const long long at = total > 0 ? (long long)((double)wid * (double)total / (double)nwarps) : 0;
        int lo = 0, hi = nq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ecum[mid] <= at) lo = mid;
            else hi = mid - 1;
        }
        home = lo;
    }
    int idle = 0, home_polls = 0;
    for (;;) {
        int pos = -1, stage = -1, item = 0, items = 0;
        if (lane == 0) {
            if (home >= 0) {
                stage = pool_claim(qs[home], &item, &items);
                if (stage >= 0) {
                    pos = home;
                    home_polls = 0;
                } else if (ld_volatile(&qs[home].live) == 0) {
                    home = -1;  // done: adopt the next query found with work
                } else {
                    ++home_polls;
                }
            }
            if (pos < 0 && (home < 0 || home_polls > kPoolHomePolls)) {
                pos = scan_and_claim(qs, nq, wid, &stage, &item, &items);
                if (pos >= 0) {
                    home_polls = 0;
                    if (home < 0) home = pos;
                }
            }
        }
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (pos < 0) {
            int stop = 0;
            if (lane == 0) stop = ld_volatile(&pool->finished) >= nq || ld_volatile(&pool->error) != 0;
            if (__shfl_sync(0xffffffffu, stop, 0)) break;
            if (++idle > kPoolIdleLimit) {
                if (lane == 0) atomicCAS(&pool->error, 0, (int)GMT_ERR_TIMEOUT);
                break;
            }
            __nanosleep(idle < 32 ? 32 : 128);
            continue;
        }
        idle = 0;
        stage = __shfl_sync(0xffffffffu, stage, 0);
        item = __shfl_sync(0xffffffffu, item, 0);
        items = __shfl_sync(0xffffffffu, items, 0);
        PoolQ& Q = qs[pos];
        const PlanArgs& A = args[order[pos]];
        // the stage's parameters, read by lane 0 after its acquiring claim
        PoolIter I;
        if (lane == 0) {
            I.it = __ldcg(&Q.iter.it);
            I.ncur = __ldcg(&Q.iter.ncur);
            I.nk = __ldcg(&Q.iter.nk);
            I.ng_prev = __ldcg(&Q.iter.ng_prev);
            I.theta = __ldcg(&Q.iter.theta);
            I.i = __ldcg(&Q.iter.i);
            I.ng = __ldcg(&Q.iter.ng);
            I.nc = __ldcg(&Q.iter.nc);
        }
        I.it = __shfl_sync(0xffffffffu, I.it, 0);
        I.ncur = __shfl_sync(0xffffffffu, I.ncur, 0);
        I.nk = __shfl_sync(0xffffffffu, I.nk, 0);
        I.ng_prev = __shfl_sync(0xffffffffu, I.ng_prev, 0);
        I.theta = __shfl_sync(0xffffffffu, I.theta, 0);
        I.i = __shfl_sync(0xffffffffu, I.i, 0);
        I.ng = __shfl_sync(0xffffffffu, I.ng, 0);
        I.nc = __shfl_sync(0xffffffffu, I.nc, 0);
        TaskCounters cnt;
        const int kk = kernel_kind(A);
        if (ALL_KINDS && kk == 0) run_item<GMT_COST_DI, 3>(A, stage, item, I, cnt);
        else if (ALL_KINDS && kk == 1) run_item<GMT_COST_DUBINS, 3>(A, stage, item, I, cnt);
        else if (kk == 2) run_item<GMT_COST_EUCLID, 2>(A, stage, item, I, cnt);
        else run_item<GMT_COST_EUCLID, 3>(A, stage, item, I, cnt);
        __syncwarp();  // every lane's writes before lane 0's releasing completion
        if (lane == 0) {
            flush_counters(A.ctl, cnt);
            if (add_acq_rel(&Q.done, 1) == items - 1) end_stage(A, Q, stage, I, pool);
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_plan_pool(const PlanArgs* args, const int* order, const long long* ecum, int nq, PoolQ* qs,
                             PoolCtl* pool, bool all_kinds, int blocks, int threads, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    pool_init_kernel<<<nq, 256, 0, st>>>(args, order, qs, pool);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (all_kinds) pool_kernel<true><<<blocks, threads, 0, st>>>(args, order, ecum, nq, qs, pool);
    else pool_kernel<false><<<blocks, threads, 0, st>>>(args, order, ecum, nq, qs, pool);
    return cudaGetLastError();
}

int plan_pool_max_blocks(int threads, bool all_kinds) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const cudaError_t e =
        all_kinds ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pool_kernel<true>, threads, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pool_kernel<false>, threads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

}  // namespace gmtk
