// Algorithm 1 (Group Marching Tree) as one persistent CUDA kernel.
//
// A "team" of threads runs every wavefront iteration of one plan without
// returning to the host: one CTA (block barriers), one thread-block cluster
// (hardware cluster barriers) or a cooperative grid (bounded global
// barriers, co-residency guaranteed by the cooperative launch).  Each
// iteration i has two phases separated by team barriers:
//
//   1  the open-set snapshot `ocost` (cost if open, +inf otherwise) is
//      brought up to date with the previous iteration (its group closed, the
//      nodes it opened set to their costs); group selection (Alg. 1's group) splits
//      the open list into G_i = {v open : cost(v) <= theta_i} and the nodes
//      that stay open; the warp that selects a node of G_i at once pushes it
//      (the frontier push): it scans the node's out-row and claims every unexplored
//      neighbour once per iteration through one atomicMax on its stamp
//      (INT_MAX marks tree nodes), appending it to the candidate list.
//      Nothing reads the snapshot in this phase.
//   2  lazy parent, check and commit: one warp per candidate x scans its in-row,
//      gathers the snapshot and takes argmin of (ocost[y] + c(y, x), y); the
//      warp checks that single edge (points spread over the lanes) and, if it
//      is free, commits parent and cost and appends x to the next open list.
//
// Open entries carry their cost, so selection and the snapshot update need
// no gathers.  Open entries are dealt to the team's CTAs round-robin first,
// then to their warps, then to lanes, so that the nodes of a small group (and
// their pushes) spread over the team.  An open list keeps the entries that
// stay open at its front and the newly opened nodes at its back, so phase 1
// of the next iteration finds exactly the nodes the snapshot lacks.
//
// After phase 2 every thread reads the same totals and decides (Alg. 1's termination test):
// success if G_i held a goal node, failure if no node stays open, else the
// next threshold index is the smallest i' > i with theta_{i'} >= min open cost
// (iterations whose group would be empty are no-ops and are skipped).  Lists
// are appended with one atomic per warp (ballot + popc prefix), the prefix-sum
// compaction of Section IV.  Counters are double-buffered by parity so that
// resets need no extra barrier.
#include "plan_core.cuh"
#include "plan_fused.cuh"

namespace gmtk {

// ------------------------------------------------------------------- kernel
// sbox_bytes: shared memory at sbox for staged boxes and, once the wavefront is
// over, the copy of the parent array.
template <class Team, int KIND, int DP, bool SM = false>
__device__ __forceinline__ void plan_body(const PlanArgs& A, const Team& team, float* sbox, size_t sbox_bytes) {
    constexpr int D = KIND == GMT_COST_DI ? 6 : (KIND == GMT_COST_DUBINS ? 4 : DP);
    const int nbs = A.boxes.count <= smem_box_cap(DP) ? A.boxes.count : 0;
    for (int t = threadIdx.x; t < nbs * DP; t += blockDim.x) {
        sbox[t] = A.boxes.lo[t];
        sbox[nbs * DP + t] = A.boxes.hi[t];
    }
    __syncthreads();
    const float* blo = nbs ? sbox : A.boxes.lo;
    const float* bhi = nbs ? sbox + nbs * DP : A.boxes.hi;
    const int nbox = A.boxes.count;

    PlanCtl* ctl = A.ctl;
    const int rank = team.rank(), size = team.size();
    // The result fields and counters start at zero here, so that a launch
    // whose barrier keeps no state in the control block needs no memset of it
    // first (the first team barrier, or the early return below, orders these
    // stores before every other access).
    if (rank == 0) {
        ctl->error = 0;
        ctl->status = 0;
        ctl->iters = ctl->final_i = ctl->path_len = 0;
        ctl->goal_node = -1;
        ctl->push_edges = ctl->pull_edges = ctl->checks = ctl->failed = ctl->tree_size = 0ull;
        ctl->checks_computed = 0ull;
    }
    if (A.check_edges) {
        const long long e = max(__ldcg(&A.out_row[A.N]), __ldcg(&A.in_row[A.N]));
        if (e > A.edge_cap) {  // uniform across the team: every thread reads the same counts
            if (rank == 0) {
                ctl->status = GMT_ERR_OOM;
                ctl->goal_node = -1;
            }
            return;
        }
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    const int gwarp = rank >> 5, nwarps = size >> 5;
    const int cta = team.cta(), nctas = team.ctas();
    const float INF = f_inf();
    const unsigned INF_KEY = 0x7f800000u;
    const int N = A.N;

    // Initialisation: x_init is the only open node and the root of the tree.
    // stamp[v]: INT_MAX once v is in the tree, else the last iteration that
    // claimed v as a candidate (-1: never)
    for (int v = rank; v < N; v += size) {
        const float c0 = v == 0 ? 0.0f : INF;
        A.cost[v] = c0;
        A.ocost[v] = c0;
        A.parent[v] = -1;
        A.stamp[v] = v == 0 ? INT_MAX : -1;
    }
    if (rank == 0) {
        A.list_open[0][0] = make_int2(0, __float_as_int(0.0f));
        for (int k = 0; k < 2; ++k) {
            ctl->gk[k] = 0ull;
            ctl->new_count[k] = ctl->cand_count[k] = 0;
            ctl->min_keep[k] = ctl->min_new[k] = INF_KEY;
            ctl->goal_flag[k] = 0;
        }
        ctl->gk[1] = 1ull << 32;  // one kept entry in open list 0
        // the minimum (cost, index) goal node of the tree so far: x_init at cost 0 if it is one
        ctl->goal_key = A.is_goal[0] ? 0ull : ~0ull;
    }
    bool ok = team.sync(ctl);

    long long i = 0;
    float theta = 0.0f;
    int it = 0;
    int status = GMT_OK;
    unsigned long long n_push = 0, n_pull = 0;       // edges: may exceed 2^32 over a dense graph
    unsigned n_checks = 0, n_failed = 0, n_computed = 0;  // per thread at most N each
    unsigned n_tree = rank == 0 ? 1u : 0u;  // tree nodes: x_init, then one per commit

    while (ok) {
        if (it >= A.max_iters) { status = GMT_ERR_ITER_LIMIT; break; }
        const int p = it & 1;
        const int2* cur = A.list_open[p];
        int2* nxt = A.list_open[p ^ 1];
        int* G = A.list_g[p];

        // ---- phase 1: snapshot update, group selection, push
        const unsigned long long gk_prev = st_ull<SM>(&ctl->gk[p ^ 1]);
        const int nk = (int)(gk_prev >> 32), nn = st_i<SM>(&ctl->new_count[p]);
        // the lane's first open entry, loaded now so that its latency overlaps
        // the snapshot update below (which writes ocost only, never cur)
        const int ncur = nk + nn;
        const int t_first = cta + nctas * wib + nctas * wpc * lane;
        int2 e_first = make_int2(-1, 0);
        if (t_first < ncur) e_first = st_i2<SM>(&cur[t_first < nk ? t_first : N - 1 - (t_first - nk)]);
        if (it > 0) {
            const int ng_prev = (int)(gk_prev & 0xffffffffu);
            const int* Gprev = A.list_g[p ^ 1];
            for (int t = rank; t < ng_prev; t += size) A.ocost[st_i<SM>(&Gprev[t])] = INF;
            for (int t = rank; t < nn; t += size) {
                const int2 e = st_i2<SM>(&cur[N - 1 - t]);
                A.ocost[e.x] = __int_as_float(e.y);
            }
        }
        {
            const int per_round = nctas * wpc * 32;
            for (int t0 = cta + nctas * wib; t0 < ncur; t0 += per_round) {  // t0: entry of lane 0
                const int t = t0 + nctas * wpc * lane;
                bool in_g = false, keep = false;
                int2 e = make_int2(-1, 0);
                if (t < ncur) {
                    e = t0 == cta + nctas * wib ? e_first : st_i2<SM>(&cur[t < nk ? t : N - 1 - (t - nk)]);
                    in_g = __int_as_float(e.y) <= theta;
                    keep = !in_g;
                }
                // one atomic reserves the warp's group entries and kept entries
                const unsigned mg = __ballot_sync(0xffffffffu, in_g), mkeep = __ballot_sync(0xffffffffu, keep);
                unsigned long long base = 0;
                if (lane == 0 && (mg | mkeep))
                    base = atomicAdd(&ctl->gk[p], ((unsigned long long)__popc(mkeep) << 32) | __popc(mg));
                base = __shfl_sync(0xffffffffu, base, 0);
                const unsigned below = (1u << lane) - 1u;
                if (in_g) {
                    G[(int)(base & 0xffffffffu) + __popc(mg & below)] = e.x;
                    if (A.is_goal[e.x]) ctl->goal_flag[p] = 1;
                }
                if (keep) nxt[(int)(base >> 32) + __popc(mkeep & below)] = e;
                const unsigned kmin =
                    __reduce_min_sync(0xffffffffu, keep ? float_key(__int_as_float(e.y)) : INF_KEY);
                if (lane == 0 && kmin != INF_KEY) atomicMin(&ctl->min_keep[p], kmin);
                for (unsigned gm = __ballot_sync(0xffffffffu, in_g); gm; gm &= gm - 1) {
                    const int z = __shfl_sync(0xffffffffu, e.x, __ffs(gm) - 1);
                    const int e0 = __ldg(&A.out_row[z]), e1 = __ldg(&A.out_row[z + 1]);
                    if (lane == 0) n_push += (unsigned long long)(e1 - e0);
                    // two chunks of 32 at a time: their column loads, their claims,
                    // and one slot reservation, each issued together
                    for (int eb = e0; eb < e1; eb += 2 * 32) {
                        int xs[2];
                        bool want[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int ei = eb + 32 * u + lane;
                            xs[u] = ei < e1 ? __ldg(&A.out_col[ei]) : -1;
                        }
#pragma unroll
                        for (int u = 0; u < 2; ++u)
                            // one atomic both tests "unexplored" (stamp < INT_MAX) and
                            // claims x for this iteration (stamp < it before)
                            want[u] = xs[u] >= 0 && atomicMax(&A.stamp[xs[u]], it) < it;
                        const unsigned m0 = __ballot_sync(0xffffffffu, want[0]);
                        const unsigned m1 = __ballot_sync(0xffffffffu, want[1]);
                        const int n0 = __popc(m0), total = n0 + __popc(m1);
                        if (total == 0) continue;
                        int slot = 0;
                        if (lane == 0) slot = atomicAdd(&ctl->cand_count[p], total);
                        slot = __shfl_sync(0xffffffffu, slot, 0);
                        const unsigned below = (1u << lane) - 1u;
                        if (want[0]) A.list_cand[slot + __popc(m0 & below)] = xs[0];
                        if (want[1]) A.list_cand[slot + n0 + __popc(m1 & below)] = xs[1];
                    }
                }
            }
        }
        if (!(ok = team.sync(ctl))) break;

        // ---- phase 2: lazy parent selection, one collision check, commit
        if (rank == 0) {
            ctl->gk[p ^ 1] = 0ull;  // previous group list, kept entries of this iteration's open list
            ctl->new_count[p] = 0;
            ctl->cand_count[p ^ 1] = 0;
            ctl->min_keep[p ^ 1] = INF_KEY;
            ctl->min_new[p ^ 1] = INF_KEY;
            ctl->goal_flag[p ^ 1] = 0;
        }
        {
            // the warp's first candidate slot, loaded with the count (the list
            // holds at least N entries; the value is used only if ci < nc)
            const int x_first = gwarp < N ? st_i<SM>(&A.list_cand[gwarp]) : -1;
            const int nc = st_i<SM>(&ctl->cand_count[p]);
            for (int ci = gwarp; ci < nc; ci += nwarps) {
                const int x = ci == gwarp ? x_first : st_i<SM>(&A.list_cand[ci]);
                const int r0 = __ldg(&A.in_row[x]), r1 = __ldg(&A.in_row[x + 1]);
                const bool x_goal = A.is_goal[x] != 0;
                float sx[D];  // issued now, used by the check after the reduction
#pragma unroll
                for (int a = 0; a < D; ++a) sx[a] = __ldg(&A.X[(size_t)a * A.pitch + x]);
                float bc;
                int by, be;
                lane_parent_min<SM>(A.in_col, A.in_cost, A.ocost, r0, r1, lane, &bc, &by, &be);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const float oc = __shfl_xor_sync(0xffffffffu, bc, off);
                    const int oy = __shfl_xor_sync(0xffffffffu, by, off);
                    const int oe = __shfl_xor_sync(0xffffffffu, be, off);
                    if (oc < bc || (oc == bc && oy < by)) { bc = oc; by = oy; be = oe; }
                }
                // The node of G that pushed x is an open in-neighbour, so be >= 0;
                // the guard only keeps a broken invariant from reading out of bounds.
                if (be < 0) {
                    if (lane == 0) { ++n_checks; ++n_failed; atomicCAS(&ctl->error, 0, (int)GMT_ERR_CUDA); }
                    continue;
                }
                float sy[D];
#pragma unroll
                for (int a = 0; a < D; ++a) sy[a] = __ldg(&A.X[(size_t)a * A.pitch + by]);
                bool free_edge;
                const int cached = A.verdict ? (int)__ldcg(&A.verdict[be]) : 0;
                if (cached != 0) {
                    free_edge = cached == 1;
                } else {
                    if (KIND == GMT_COST_EUCLID)
                        free_edge = segment_free_warp<DP>(sy, sx, __ldg(&A.in_cost[be]), A.seg_spacing, blo, bhi,
                                                          nbox, A.grid);
                    else if (KIND == GMT_COST_DUBINS) {
                        // the edge's shortest word: stored by the graph build, or recomputed
                        DubPath P;
                        if (A.in_path) {
                            const float4 w = __ldg(reinterpret_cast<const float4*>(A.in_path) + be);
                            P = DubPath{__float_as_int(w.w), w.x, w.y, w.z, ((w.x + w.y) + w.z) * A.rho};
                        } else {
                            P = dubins_path(sy, sx, A.rho);
                        }
                        free_edge = dubins_free_warp(sy, sx, P, __ldg(&A.in_cost[be]), A.seg_spacing, A.rho,
                                                     A.pos_lo, A.pos_hi, blo, bhi, nbox, A.grid);
                    }
                    else {
                        // arrival time of the edge: stored by the graph build, or recomputed
                        const float tau = A.in_tau ? __ldg(&A.in_tau[be]) : di_tau(di_coef(sy, sx), A.r);
                        free_edge = trajectory_free_warp(sy, sx, tau, A.traj_points, A.pos_lo, A.pos_hi, blo, bhi, nbox,
                                                         A.grid);
                    }
                    if (lane == 0) {
                        ++n_computed;
                        if (A.verdict) A.verdict[be] = free_edge ? 1 : 2;
                    }
                }
                if (lane == 0) {
                    n_pull += (unsigned long long)(r1 - r0);
                    ++n_checks;
                    if (free_edge) {
                        A.cost[x] = bc;
                        A.parent[x] = by;
                        A.stamp[x] = INT_MAX;
                        const int s = atomicAdd(&ctl->new_count[p ^ 1], 1);
                        nxt[N - 1 - s] = make_int2(x, __float_as_int(bc));
                        atomicMin(&ctl->min_new[p], float_key(bc));
                        // a tree node's cost never changes, so the minimum goal
                        // node over commits is the returned path's minimum over the tree
                        ++n_tree;
                        if (x_goal) atomicMin(&ctl->goal_key, ((unsigned long long)float_key(bc) << 32) | (unsigned)x);
                    } else {
                        ++n_failed;
                    }
                }
            }
        }
        if (!(ok = team.sync(ctl))) break;

        // ---- termination test, next threshold
        const int goal = st_i<SM>(&ctl->goal_flag[p]);
        const int n_open = (int)(st_ull<SM>(&ctl->gk[p]) >> 32) + st_i<SM>(&ctl->new_count[p ^ 1]);
        const unsigned mk = min(st_u<SM>(&ctl->min_keep[p]), st_u<SM>(&ctl->min_new[p]));
        ++it;
        if (goal) { status = GMT_OK; break; }
        if (n_open == 0) { status = GMT_NO_PATH; break; }
        const float m = __uint_as_float(mk);
        if (A.delta == 0.0f) {
            theta = m;
            i = i + 1;
        } else {
            const float qk = m / A.delta;
            if (!(qk < 16777216.0f)) { status = GMT_ERR_ITER_LIMIT; break; }  // i stays below 2^24
            long long k = (long long)ceilf(qk);
            if (k < i + 1) k = i + 1;
            while (k > i + 1 && (float)(k - 1) * A.delta >= m) --k;
            while ((float)k * A.delta < m) ++k;
            i = k;
            theta = (float)i * A.delta;
        }
    }

    // ---- result: counters (the goal node was tracked at each commit; the loop
    // ended after a team barrier, so every commit is visible), path
    if (ok) {
        unsigned long long checks = n_checks, failed = n_failed, computed = n_computed, tree = n_tree;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            n_push += __shfl_xor_sync(0xffffffffu, n_push, off);
            n_pull += __shfl_xor_sync(0xffffffffu, n_pull, off);
            checks += __shfl_xor_sync(0xffffffffu, checks, off);
            failed += __shfl_xor_sync(0xffffffffu, failed, off);
            computed += __shfl_xor_sync(0xffffffffu, computed, off);
            tree += __shfl_xor_sync(0xffffffffu, tree, off);
        }
        if (lane == 0) {
            atomicAdd(&ctl->push_edges, n_push);
            atomicAdd(&ctl->pull_edges, n_pull);
            atomicAdd(&ctl->checks, checks);
            atomicAdd(&ctl->failed, failed);
            atomicAdd(&ctl->checks_computed, computed);
            atomicAdd(&ctl->tree_size, tree);
        }
    }
    // The returned path is walked by rank 0 from the goal node back to x_init.
    // The wavefront is over and the staged boxes are no longer needed, so CTA 0
    // first copies the parent array into that shared memory when it fits:
    // each hop is then a shared-memory read instead of an L2 round trip.
    int* const spar = reinterpret_cast<int*>(sbox);
    const bool par_in_smem = ok && status == GMT_OK && (size_t)N * sizeof(int) <= sbox_bytes;
    if (par_in_smem && team.cta() == 0) {  // uniform over CTA 0
        for (int v = threadIdx.x; v < N; v += blockDim.x) spar[v] = ldcg_i(&A.parent[v]);
        __syncthreads();
    }
    if (rank == 0) {
        const int err = ld_volatile(&ctl->error);
        ctl->status = err ? err : status;
        ctl->iters = it;
        ctl->final_i = (int)i;
        ctl->goal_node = -1;
        ctl->path_len = 0;
        if (ok && status == GMT_OK) {
            const int g = (int)(ctl->goal_key & 0xffffffffu);
            ctl->goal_node = g;
            auto parent_of = [&](int v) { return par_in_smem ? spar[v] : ldcg_i(&A.parent[v]); };
            int len = 1, v = g;
            while (v > 0 && len <= N) {
                v = parent_of(v);
                ++len;
            }
            if (v != 0) len = 0;  // not a chain back to x_init: report no path
            ctl->path_len = len;
            if (A.path) {
                v = g;
                for (int k = len - 1; k >= 0; --k) {
                    A.path[k] = v;
                    if (v > 0) v = parent_of(v);
                }
            }
        }
    }
}

// The first warp copies the final control block to the caller's mapped host
// copy (src: a block whose writers have all passed a barrier since).
__device__ __forceinline__ void publish_ctl(PlanCtl* dst, const PlanCtl* src, int rank) {
    constexpr int n = (int)(sizeof(PlanCtl) / sizeof(int));
    for (int t = rank; t < n; t += 32)
        reinterpret_cast<int*>(dst)[t] = __ldcg(reinterpret_cast<const int*>(src) + t);
}

// Lanes per candidate pull (measured on one GB300): a single plan's team has
// hundreds of warps for a frontier of a few hundred candidates, and 16-lane
// pulls only lengthen each candidate's chain (DI n = 4096: 0.209 against
// 0.132 ms); a batch's 4-CTA teams see more candidates per warp, and two
// 16-lane pulls per warp take the 256-query plan stage from 2.41 to 2.26 ms.
constexpr int kPlanPullLanes = 32;
constexpr int kBatchPullLanes = 16;

// One plan on a team that spans several SMs (or one CTA whose state does not
// fit its shared memory): the one-barrier wavefront (A.ocost holds 2 N floats).
template <class Team, int KIND, int DP>
__global__ void __launch_bounds__(1024, 1) plan_kernel(PlanArgs A, Team team) {
    extern __shared__ float sbox[];
    unsigned dyn_smem;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
    plan_body_fused<Team, KIND, DP, kPlanPullLanes>(A, team, sbox, dyn_smem);
    if (A.host_ctl) {
        team.sync(A.ctl);  // every warp's counters and rank 0's result are in
        if (team.rank() < 32) publish_ctl(A.host_ctl, A.ctl, team.rank());
    }
}

// One CTA whose wavefront state lives in its shared memory: after the region
// of staged boxes / parent copy (region0 bytes) come the control block, the
// snapshot (ocost), the stamps and the lists (plan_smem_state_bytes).  Every
// step of the body then touches L2 only for the read-only CSR, the samples and
// the outputs.  The control block is copied out for the host at the end.
template <int KIND, int DP>
__global__ void __launch_bounds__(1024, 1) plan_kernel_smem(PlanArgs A, unsigned region0) {
    extern __shared__ __align__(16) float smem[];
    unsigned char* base = reinterpret_cast<unsigned char*>(smem);
    PlanCtl* gctl = A.ctl;
    PlanCtl* sctl = reinterpret_cast<PlanCtl*>(base + region0);
    const size_t N = (size_t)A.N;
    float* socost = reinterpret_cast<float*>(base + region0 + kSmemCtlBytes);
    int* sstamp = reinterpret_cast<int*>(socost + N);
    int* slists = reinterpret_cast<int*>(base + region0 + kSmemCtlBytes + smem_round16(8 * N));
    for (int t = threadIdx.x; t < (int)(sizeof(PlanCtl) / sizeof(int)); t += blockDim.x)
        reinterpret_cast<int*>(sctl)[t] = 0;
    __syncthreads();
    A.ctl = sctl;
    A.ocost = socost;
    A.stamp = sstamp;
    assign_plan_lists(A, slists, N);
    plan_body<BlockTeam, KIND, DP, true>(A, BlockTeam{}, smem, region0);
    __syncthreads();
    for (int t = threadIdx.x; t < (int)(sizeof(PlanCtl) / sizeof(int)); t += blockDim.x) {
        const int v = reinterpret_cast<const int*>(sctl)[t];
        reinterpret_cast<int*>(gctl)[t] = v;
        if (A.host_ctl) reinterpret_cast<int*>(A.host_ctl)[t] = v;
    }
}

// Persistent batched wavefront: every team (a CTA, or a cluster) takes the next
// query from a device queue (every query of the batch, of any kind, ordered by
// decreasing size), runs the one-barrier wavefront on it with its own scratch
// slice, and repeats until the queue is empty.  Queries never wait for each
// other, so teams need no co-scheduling beyond their own CTAs.  ALL_KINDS =
// false: a lean instantiation for batches of geometric queries only.
template <class Team, bool ALL_KINDS>
__global__ void __launch_bounds__(1024, 1) plan_batch_kernel(const PlanArgs* __restrict__ queries,
                                                          const int* __restrict__ order, int nq,
                                                          int* __restrict__ next, int* __restrict__ slot,
                                                          BatchScratch scratch, Team team) {
    extern __shared__ float sbox[];
    const int team_id = team.id();
    for (;;) {
        if (team.rank() == 0) slot[team_id] = atomicAdd(next, 1);
        team.sync(nullptr);
        const int k = __ldcg(&slot[team_id]);
        if (k >= nq) break;
        PlanArgs A = queries[order[k]];
        const size_t nm = (size_t)scratch.max_nodes;
        A.ocost = scratch.ocost + team_id * 2 * nm;
        A.stamp = scratch.stamp + team_id * nm;
        assign_plan_lists(A, scratch.lists + team_id * plan_list_stride(nm), nm);
        unsigned dyn_smem;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
        // counters in the control block: in this kernel (four bodies inlined)
        // the shared copy cost registers and measured no faster
        constexpr int W = kBatchPullLanes;
        constexpr bool SH = false;
        if (ALL_KINDS && A.kind == GMT_COST_DI) plan_body_fused<Team, GMT_COST_DI, 3, W, SH>(A, team, sbox, dyn_smem);
        else if (ALL_KINDS && A.kind == GMT_COST_DUBINS)
            plan_body_fused<Team, GMT_COST_DUBINS, 3, W, SH>(A, team, sbox, dyn_smem);
        else if (A.dp == 2) plan_body_fused<Team, GMT_COST_EUCLID, 2, W, SH>(A, team, sbox, dyn_smem);
        else plan_body_fused<Team, GMT_COST_EUCLID, 3, W, SH>(A, team, sbox, dyn_smem);
        team.sync(nullptr);
    }
}

// Persistent batched wavefront with one CTA per query whose state lives in
// its shared memory (the batch's one-CTA teams when the largest query fits):
// the CTA takes the next query from the device queue and runs the body of
// plan_kernel_smem on it (control block, snapshot, stamps and lists after
// region0 bytes of staged boxes / parent copy), then copies the control block
// out.
template <bool ALL_KINDS>
__global__ void __launch_bounds__(1024, 1) plan_batch_smem_kernel(const PlanArgs* __restrict__ queries,
                                                               const int* __restrict__ order, int nq,
                                                               int* __restrict__ next, unsigned region0) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int kq;
    unsigned char* base = reinterpret_cast<unsigned char*>(smem);
    PlanCtl* sctl = reinterpret_cast<PlanCtl*>(base + region0);
    for (;;) {
        if (threadIdx.x == 0) kq = atomicAdd(next, 1);
        __syncthreads();
        const int k = kq;
        if (k >= nq) break;
        PlanArgs A = queries[order[k]];
        const size_t N = (size_t)A.N;
        PlanCtl* gctl = A.ctl;
        float* socost = reinterpret_cast<float*>(base + region0 + kSmemCtlBytes);
        int* sstamp = reinterpret_cast<int*>(socost + N);
        int* slists = reinterpret_cast<int*>(base + region0 + kSmemCtlBytes + smem_round16(8 * N));
        for (int t = threadIdx.x; t < (int)(sizeof(PlanCtl) / sizeof(int)); t += blockDim.x)
            reinterpret_cast<int*>(sctl)[t] = 0;
        __syncthreads();
        A.ctl = sctl;
        A.ocost = socost;
        A.stamp = sstamp;
        assign_plan_lists(A, slists, N);
        if (ALL_KINDS && A.kind == GMT_COST_DI) plan_body<BlockTeam, GMT_COST_DI, 3, true>(A, BlockTeam{}, smem, region0);
        else if (ALL_KINDS && A.kind == GMT_COST_DUBINS)
            plan_body<BlockTeam, GMT_COST_DUBINS, 3, true>(A, BlockTeam{}, smem, region0);
        else if (A.dp == 2) plan_body<BlockTeam, GMT_COST_EUCLID, 2, true>(A, BlockTeam{}, smem, region0);
        else plan_body<BlockTeam, GMT_COST_EUCLID, 3, true>(A, BlockTeam{}, smem, region0);
        __syncthreads();
        for (int t = threadIdx.x; t < (int)(sizeof(PlanCtl) / sizeof(int)); t += blockDim.x)
            reinterpret_cast<int*>(gctl)[t] = reinterpret_cast<const int*>(sctl)[t];
        __syncthreads();  // the next query reuses the shared memory
    }
}

// ----------------------------------------------------------------- launcher
namespace {
template <int KIND, int DP>
cudaError_t plan_t(const PlanArgs& a, int blocks, int threads, int cluster, cudaStream_t st) {
    const int nbs = a.boxes.count <= smem_box_cap(DP) ? a.boxes.count : 0;
    const size_t smem = plan_smem_bytes(nbs, DP, a.N);
    if (cluster > 1) {
        auto kern = plan_kernel<ClusterTeam, KIND, DP>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cluster);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, a, ClusterTeam{});
    }
    if (blocks <= 1) {
        // one CTA: the wavefront state goes to shared memory when it fits
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t region0 = smem_round16(smem);
        const size_t total = plan_smem_state_bytes(region0, a.N);
        if (total <= (size_t)optin) {
            auto kern = plan_kernel_smem<KIND, DP>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total);
            if (e != cudaSuccess) return e;
            kern<<<1, threads, total, st>>>(a, (unsigned)region0);
            return cudaGetLastError();
        }
        plan_kernel<BlockTeam, KIND, DP><<<1, threads, smem, st>>>(a, BlockTeam{});
        return cudaGetLastError();
    }
    GridTeam team;
    team.expected = (unsigned)blocks + ((a.debug_flags & GMT_DEBUG_UNREACHABLE_BARRIER) ? 1u : 0u);
    team.spin_limit = a.spin_limit > 0 ? a.spin_limit : kDefaultSpinLimit;
    PlanArgs args = a;
    void* params[] = {&args, &team};
    return cudaLaunchCooperativeKernel((const void*)plan_kernel<GridTeam, KIND, DP>, dim3(blocks), dim3(threads),
                                       params, smem, st);
}

template <int KIND, int DP>
int occupancy_t(int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = plan_smem_bytes(smem_box_cap(DP), DP, 12 * 1024);  // the most a launch asks for
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_kernel<GridTeam, KIND, DP>, threads, smem);
    return per_sm * sms;
}
}  // namespace

cudaError_t launch_plan(const PlanArgs& a, int blocks, int threads, cudaStream_t st, int cluster) {
    if (a.kind == GMT_COST_DI) return plan_t<GMT_COST_DI, 3>(a, blocks, threads, cluster, st);
    if (a.kind == GMT_COST_DUBINS) return plan_t<GMT_COST_DUBINS, 3>(a, blocks, threads, cluster, st);
    switch (a.dp) {
        case 2: return plan_t<GMT_COST_EUCLID, 2>(a, blocks, threads, cluster, st);
        case 3: return plan_t<GMT_COST_EUCLID, 3>(a, blocks, threads, cluster, st);
        case 4: return plan_t<GMT_COST_EUCLID, 4>(a, blocks, threads, cluster, st);
        case 5: return plan_t<GMT_COST_EUCLID, 5>(a, blocks, threads, cluster, st);
        case 6: return plan_t<GMT_COST_EUCLID, 6>(a, blocks, threads, cluster, st);
        case 7: return plan_t<GMT_COST_EUCLID, 7>(a, blocks, threads, cluster, st);
        case 8: return plan_t<GMT_COST_EUCLID, 8>(a, blocks, threads, cluster, st);
        case 9: return plan_t<GMT_COST_EUCLID, 9>(a, blocks, threads, cluster, st);
        case 10: return plan_t<GMT_COST_EUCLID, 10>(a, blocks, threads, cluster, st);
        default: return cudaErrorInvalidValue;
    }
}

// Largest cluster size (16, 8, 4, 2) for which one cluster of `threads`-thread
// CTAs of the plan kernel can be resident; 0 if none.
int plan_max_cluster(int kind, int dp, int threads) {
    auto kern = kind == GMT_COST_DI       ? plan_kernel<ClusterTeam, GMT_COST_DI, 3>
                : kind == GMT_COST_DUBINS ? plan_kernel<ClusterTeam, GMT_COST_DUBINS, 3>
                : dp == 2                 ? plan_kernel<ClusterTeam, GMT_COST_EUCLID, 2>
                                          : plan_kernel<ClusterTeam, GMT_COST_EUCLID, 3>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
    for (int c = 16; c >= 2; c /= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = plan_smem_bytes(smem_box_cap(3), 3, 12 * 1024);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0) return c;
    }
    cudaGetLastError();
    return 0;
}

namespace {
template <bool ALL_KINDS>
cudaError_t plan_batch_t(const PlanArgs* queries, const int* order, int nq, int* next, int* slot,
                         const BatchScratch& scratch, int teams, int threads, int cluster, size_t smem,
                         int max_n, cudaStream_t st) {
    if (cluster <= 1 && batch_state_fits(smem, max_n)) {
        const size_t region0 = smem_round16(smem), total = plan_smem_state_bytes(region0, max_n);
        auto kern = plan_batch_smem_kernel<ALL_KINDS>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total);
        if (e != cudaSuccess) return e;
        kern<<<teams, threads, total, st>>>(queries, order, nq, next, (unsigned)region0);
        return cudaGetLastError();
    }
    if (cluster <= 1) {
        auto kern = plan_batch_kernel<BlockTeam, ALL_KINDS>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<teams, threads, smem, st>>>(queries, order, nq, next, slot, scratch, BlockTeam{});
        return cudaGetLastError();
    }
    auto kern = plan_batch_kernel<ClusterTeam, ALL_KINDS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(teams * cluster);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, queries, order, nq, next, slot, scratch, ClusterTeam{});
}

template <bool ALL_KINDS>
int batch_teams_t(int threads, int cluster, size_t smem, int max_n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cluster <= 1 && batch_state_fits(smem, max_n)) {
        const size_t total = plan_smem_state_bytes(smem_round16(smem), max_n);
        auto kern = plan_batch_smem_kernel<ALL_KINDS>;
        int per_sm = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, total) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return per_sm * sms;
    }
    if (cluster <= 1) {
        auto kern = plan_batch_kernel<BlockTeam, ALL_KINDS>;
        int per_sm = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return per_sm * sms;
    }
    auto kern = plan_batch_kernel<ClusterTeam, ALL_KINDS>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}
}  // namespace

cudaError_t launch_plan_batch(const PlanArgs* queries, const int* order, int nq, int* next, int* slot,
                              const BatchScratch& scratch, int teams, int threads, int cluster, size_t smem,
                              int max_n, bool all_kinds, cudaStream_t st) {
    return all_kinds ? plan_batch_t<true>(queries, order, nq, next, slot, scratch, teams, threads, cluster, smem,
                                          max_n, st)
                     : plan_batch_t<false>(queries, order, nq, next, slot, scratch, teams, threads, cluster, smem,
                                           max_n, st);
}

int plan_batch_max_teams(int threads, int cluster, size_t smem, int max_n, bool smem_state, bool all_kinds) {
    const int mn = smem_state ? max_n : INT_MAX;  // INT_MAX nodes never fit: the scratch kernels
    return all_kinds ? batch_teams_t<true>(threads, cluster, smem, mn) : batch_teams_t<false>(threads, cluster, smem, mn);
}

bool batch_state_fits(size_t smem, int max_n) {
    if (max_n <= 0 || max_n > (1 << 24)) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return plan_smem_state_bytes(smem_round16(smem), max_n) + kPlanStaticSmem <= (size_t)optin;
}

int plan_max_coresident_blocks(int kind, int dp, int threads) {
    if (kind == GMT_COST_DI) return occupancy_t<GMT_COST_DI, 3>(threads);
    if (kind == GMT_COST_DUBINS) return occupancy_t<GMT_COST_DUBINS, 3>(threads);
    switch (dp) {
        case 2: return occupancy_t<GMT_COST_EUCLID, 2>(threads);
        case 3: return occupancy_t<GMT_COST_EUCLID, 3>(threads);
        case 4: return occupancy_t<GMT_COST_EUCLID, 4>(threads);
        case 5: return occupancy_t<GMT_COST_EUCLID, 5>(threads);
        case 6: return occupancy_t<GMT_COST_EUCLID, 6>(threads);
        case 7: return occupancy_t<GMT_COST_EUCLID, 7>(threads);
        case 8: return occupancy_t<GMT_COST_EUCLID, 8>(threads);
        case 9: return occupancy_t<GMT_COST_EUCLID, 9>(threads);
        case 10: return occupancy_t<GMT_COST_EUCLID, 10>(threads);
        default: return 0;
    }
}

}  // namespace gmtk
