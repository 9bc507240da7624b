// Algorithm 1 with one team barrier per iteration (the batched teams scheme).
//
// The open-set snapshot is double-buffered: iteration i reads buffer i & 1
// (V_open as it stood when the iteration began, Sec. III-A) and builds the
// snapshot of iteration i + 1 in the other buffer, which still holds that of
// iteration i - 1: the previous group closes, the nodes opened in i - 1 open
// (unless they join G_i), G_i closes, and each commit opens its node.  Since
// nothing in iteration i changes the buffer it reads, a candidate can choose
// its lazy parent, have its one edge checked and be committed as soon as it
// is claimed: group selection, push, lazy parent, check and commit run in one
// phase, and a single team barrier ends the iteration.  Claimed candidates go
// to a team-wide queue (entries hold -1 until written); each warp pushes its
// share of the group, then takes queued candidates one ticket at a time until
// every warp has finished pushing and the queue is empty, so the pulls spread
// over the team while the last pushes are still running.  The termination
// test then reads the iteration's counters; they come in three sets
// (iteration i uses set i % 3 and resets set (i + 1) % 3, last read two
// barriers earlier), so no second barrier is needed for resets.
//
// Results, counters and the returned path are those of plan_body (the order
// in which candidates are handled does not change any decision: each lazy
// parent is the minimum (cost, index) over the snapshot).
#pragma once

#include "plan_core.cuh"

namespace gmtk {

// Shared memory of the fused body, one allocation per kernel however many
// instantiations of the body it inlines: the copy of the team's counters
// (read by the team through the cluster's shared window) and the counters of
// the termination test shared within a CTA.
static __shared__ PlanCtl fused_team_ctl;
static __shared__ unsigned fused_term[5];

struct FusedCounts {
    unsigned long long push = 0, pull = 0;
    unsigned checks = 0, failed = 0, computed = 0, tree = 0;
};

// Lazy parent (minimum (cost, index) over x's in-neighbours open in the
// snapshot ocur), one collision check of that edge, and, if it is free, the
// commit: x joins the tree and opens in the next snapshot.  One group of W
// lanes (the whole warp, or half of it: then the warp's two halves pull two
// candidates side by side).
template <int KIND, int DP, int W, bool SH>
__device__ __forceinline__ void fused_pull(const PlanArgs& A, const TeamCtl<SH>& tc, int x, const float* ocur,
                                           float* onext, int2* nxt, int set, int p, const float* blo,
                                           const float* bhi, int nbox, FusedCounts& cnt) {
    constexpr int D = KIND == GMT_COST_DI ? 6 : (KIND == GMT_COST_DUBINS ? 4 : DP);
    using LG = LaneGroup<W>;
    const int lane = LG::lane();
    const unsigned gmask = LG::mask();
    PlanCtl* ctl = A.ctl;
    const int N = A.N;
    const int r0 = __ldg(&A.in_row[x]), r1 = __ldg(&A.in_row[x + 1]);
    const bool x_goal = A.is_goal[x] != 0;
    float sx[D];
#pragma unroll
    for (int a = 0; a < D; ++a) sx[a] = __ldg(&A.X[(size_t)a * A.pitch + x]);
    float bc;
    int by, be;
    lane_parent_min<false, W>(A.in_col, A.in_cost, ocur, r0, r1, lane, &bc, &by, &be);
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        const float oc = __shfl_xor_sync(gmask, bc, off);
        const int oy = __shfl_xor_sync(gmask, by, off);
        const int oe = __shfl_xor_sync(gmask, be, off);
        if (oc < bc || (oc == bc && oy < by)) { bc = oc; by = oy; be = oe; }
    }
    // the group node that pushed x is an open in-neighbour, so be >= 0; the
    // guard keeps a broken invariant from reading out of bounds
    if (be < 0) {
        if (lane == 0) { ++cnt.checks; ++cnt.failed; tc.cas(&ctl->error, 0, (int)GMT_ERR_CUDA); }
        return;
    }
    float sy[D];
#pragma unroll
    for (int a = 0; a < D; ++a) sy[a] = __ldg(&A.X[(size_t)a * A.pitch + by]);
    bool free_edge;
    const int cached = A.verdict ? (int)__ldcg(&A.verdict[be]) : 0;
    if (cached != 0) {
        free_edge = cached == 1;
    } else {
        if (KIND == GMT_COST_EUCLID) {
            free_edge =
                segment_free_warp<DP, W>(sy, sx, __ldg(&A.in_cost[be]), A.seg_spacing, blo, bhi, nbox, A.grid);
        } else if (KIND == GMT_COST_DUBINS) {
            DubPath P;
            if (A.in_path) {
                const float4 w = __ldg(reinterpret_cast<const float4*>(A.in_path) + be);
                P = DubPath{__float_as_int(w.w), w.x, w.y, w.z, ((w.x + w.y) + w.z) * A.rho};
            } else {
                P = dubins_path(sy, sx, A.rho);
            }
            free_edge = dubins_free_warp<W>(sy, sx, P, __ldg(&A.in_cost[be]), A.seg_spacing, A.rho, A.pos_lo,
                                            A.pos_hi, blo, bhi, nbox, A.grid);
        } else {
            const float tau = A.in_tau ? __ldg(&A.in_tau[be]) : di_tau(di_coef(sy, sx), A.r);
            free_edge =
                trajectory_free_warp<W>(sy, sx, tau, A.traj_points, A.pos_lo, A.pos_hi, blo, bhi, nbox, A.grid);
        }
        if (lane == 0) {
            ++cnt.computed;
            if (A.verdict) A.verdict[be] = free_edge ? 1 : 2;
        }
    }
    if (lane == 0) {
        cnt.pull += (unsigned long long)(r1 - r0);
        ++cnt.checks;
        if (free_edge) {
            A.cost[x] = bc;
            A.parent[x] = by;
            A.stamp[x] = INT_MAX;
            onext[x] = bc;
            const int s = tc.add(&ctl->new3[set], 1);
            nxt[N - 1 - s] = make_int2(x, __float_as_int(bc));
            tc.min(&ctl->min_new3[set], float_key(bc));
            ++cnt.tree;
            if (x_goal) tc.min(&ctl->goal_key, ((unsigned long long)float_key(bc) << 32) | (unsigned)x);
        } else {
            ++cnt.failed;
        }
    }
    (void)p;
}

// sbox_bytes: shared memory at sbox for staged boxes and, once the wavefront is
// over, the copy of the parent array.  A.ocost holds 2 N floats.  W: lanes
// per candidate pull (32, or 16 for two pulls per warp).  SH: the team's
// counters in a copy in CTA 0's shared memory (a CTA or a cluster) rather
// than in the control block.
template <class Team, int KIND, int DP, int W = 32, bool SH = Team::kSharedCtl>
__device__ __forceinline__ void plan_body_fused(const PlanArgs& A, const Team& team, float* sbox, size_t sbox_bytes) {
    static_assert(!SH || Team::kSharedCtl, "shared counters need a CTA or a cluster team");
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
    // the team's counters: a copy in CTA 0's shared memory for a CTA or a
    // cluster, else the control block
    const TeamCtl<SH> tc{ctl, SH ? cluster_map(&fused_team_ctl, 0) : 0u};
    const int rank = team.rank(), size = team.size();
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
    const int cta = team.cta(), nctas = team.ctas();
    const float INF = f_inf();
    const unsigned INF_KEY = 0x7f800000u;
    const int N = A.N;
    const unsigned nwarps = (unsigned)(size >> 5);
    const int spin_limit = A.spin_limit > 0 ? A.spin_limit : kDefaultSpinLimit;

    // Initialisation: x_init is the only open node and the root of the tree;
    // both snapshot buffers hold the initial open set.
    for (int v = rank; v < N; v += size) {
        const float c0 = v == 0 ? 0.0f : INF;
        A.cost[v] = c0;
        A.ocost[v] = c0;
        A.ocost[(size_t)N + v] = c0;
        A.parent[v] = -1;
        A.stamp[v] = v == 0 ? INT_MAX : -1;
        A.list_cand[v] = -1;
    }
    if (rank == 0) {
        A.list_open[0][0] = make_int2(0, __float_as_int(0.0f));
        tc.st(&ctl->error, 0);
        for (int k = 0; k < 2; ++k) {
            tc.st(&ctl->cand_count[k], 0);
            tc.st(&ctl->ticket[k], 0);
            tc.st(&ctl->pushed[k], 0u);
        }
        for (int k = 0; k < 3; ++k) {
            tc.st(&ctl->gk3[k], 0ull);
            tc.st(&ctl->new3[k], 0);
            tc.st(&ctl->min_keep3[k], INF_KEY);
            tc.st(&ctl->min_new3[k], INF_KEY);
            tc.st(&ctl->goal3[k], 0);
        }
        tc.st(&ctl->goal_key, A.is_goal[0] ? 0ull : ~0ull);
    }
    bool ok = team.sync(ctl);

    long long i = 0;
    float theta = 0.0f;
    int it = 0;
    int status = GMT_OK;
    int nk = 1, nn = 0, ng_prev = 0;  // the open list: kept entries, newly opened entries; previous group
    FusedCounts cnt;
    unsigned n_tree = rank == 0 ? 1u : 0u;  // x_init

    while (ok) {
        if (it >= A.max_iters) { status = GMT_ERR_ITER_LIMIT; break; }
        const int p = it & 1, set = it % 3, set1 = (it + 1) % 3;
        const int2* cur = A.list_open[p];
        int2* nxt = A.list_open[p ^ 1];
        int* G = A.list_g[p];
        const int* Gprev = A.list_g[p ^ 1];
        const float* ocur = A.ocost + (size_t)p * N;
        float* onext = A.ocost + (size_t)(p ^ 1) * N;
        if (rank == 0) {
            tc.st(&ctl->gk3[set1], 0ull);
            tc.st(&ctl->new3[set1], 0);
            tc.st(&ctl->min_keep3[set1], INF_KEY);
            tc.st(&ctl->min_new3[set1], INF_KEY);
            tc.st(&ctl->goal3[set1], 0);
            // the next iteration's queue (its previous user, iteration i - 1,
            // finished with it before the last barrier)
            tc.st(&ctl->cand_count[p ^ 1], 0);
            tc.st(&ctl->ticket[p ^ 1], 0);
            tc.st(&ctl->pushed[p ^ 1], 0u);
        }
        // the previous group is closed from the next iteration on (it still
        // was open in the buffer being rebuilt)
        for (int t = rank; t < ng_prev; t += size) onext[__ldcg(&Gprev[t])] = INF;
        const int ncur = nk + nn;
        const int per_round = nctas * wpc * 32;
        for (int t0 = cta + nctas * wib; t0 < ncur; t0 += per_round) {  // t0: entry of lane 0
            const int t = t0 + nctas * wpc * lane;
            bool in_g = false, keep = false;
            int2 e = make_int2(-1, 0);
            int row0 = 0, row1 = 0;  // out-row of a group node, loaded while the warp reserves its slots
            if (t < ncur) {
                e = __ldcg(&cur[t < nk ? t : N - 1 - (t - nk)]);
                in_g = __int_as_float(e.y) <= theta;
                keep = !in_g;
                if (in_g) {
                    row0 = __ldg(&A.out_row[e.x]);
                    row1 = __ldg(&A.out_row[e.x + 1]);
                    onext[e.x] = INF;                                  // G_i closes
                } else if (t >= nk) {
                    onext[e.x] = __int_as_float(e.y);                  // opened in i - 1, stays open
                }
                if (in_g && A.is_goal[e.x]) tc.st(&ctl->goal3[set], 1);
            }
            const unsigned mg = __ballot_sync(0xffffffffu, in_g), mkeep = __ballot_sync(0xffffffffu, keep);
            const unsigned below = (1u << lane) - 1u;
            if (mg | mkeep) {
                unsigned long long base = 0;
                if (lane == 0)
                    base = tc.add(&ctl->gk3[set], ((unsigned long long)__popc(mkeep) << 32) | __popc(mg));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (in_g) G[(int)(base & 0xffffffffu) + __popc(mg & below)] = e.x;
                if (keep) nxt[(int)(base >> 32) + __popc(mkeep & below)] = e;
                const unsigned kmin =
                    __reduce_min_sync(0xffffffffu, keep ? float_key(__int_as_float(e.y)) : INF_KEY);
                if (lane == 0 && kmin != INF_KEY) tc.min(&ctl->min_keep3[set], kmin);
            }
            // push each group node of the warp: its unexplored out-neighbours are
            // claimed for this iteration and queued
            for (unsigned gm = mg; gm; gm &= gm - 1) {
                const int src = __ffs(gm) - 1;
                const int e0 = __shfl_sync(0xffffffffu, row0, src), e1 = __shfl_sync(0xffffffffu, row1, src);
                if (lane == 0) cnt.push += (unsigned long long)(e1 - e0);
                for (int eb = e0; eb < e1; eb += 4 * 32) {
                    int xs[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int ei = eb + 32 * c + lane;
                        xs[c] = ei < e1 ? __ldg(&A.out_col[ei]) : -1;
                    }
                    int st[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) st[c] = xs[c] >= 0 ? __ldcg(&A.stamp[xs[c]]) : INT_MAX;
                    unsigned m[4];
                    int total = 0;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        // stamps only grow, so one already >= it (a tree node, or one
                        // claimed this iteration) is final; else one atomic both tests
                        // "unexplored" and claims it for this iteration
                        m[c] = __ballot_sync(0xffffffffu, st[c] < it && atomicMax(&A.stamp[xs[c]], it) < it);
                        total += __popc(m[c]);
                    }
                    if (total == 0) continue;
                    int slot = 0;
                    if (lane == 0) slot = tc.add(&ctl->cand_count[p], total);
                    slot = __shfl_sync(0xffffffffu, slot, 0);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if ((m[c] >> lane) & 1u) st_volatile_i(&A.list_cand[slot + __popc(m[c] & below)], xs[c]);
                        slot += __popc(m[c]);
                    }
                }
            }
        }
        // this warp has queued all its candidates; now it pulls queued ones
        // (one ticket each) until every warp has pushed and the queue is empty
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            tc.add(&ctl->pushed[p], 1u);
        }
        for (;;) {
            int x = -1;
            if ((lane & (W - 1)) == 0) {
                const int t = tc.add(&ctl->ticket[p], 1);
                if (t < N) {
                    for (int spins = 0;; ++spins) {
                        x = ld_volatile(&A.list_cand[t]);
                        if (x >= 0) break;
                        // the queue is complete once every warp has pushed
                        if (tc.ld_acq(&ctl->pushed[p]) == nwarps && t >= tc.ld(&ctl->cand_count[p])) break;
                        if (spins > spin_limit) {
                            tc.cas(&ctl->error, 0, (int)GMT_ERR_TIMEOUT);
                            break;
                        }
                        __nanosleep(32);
                    }
                    if (x >= 0) A.list_cand[t] = -1;  // free for a later iteration
                }
            }
            x = __shfl_sync(LaneGroup<W>::mask(), x, 0, W);
            if (x < 0) break;
            fused_pull<KIND, DP, W, SH>(A, tc, x, ocur, onext, nxt, set, p, blo, bhi, nbox, cnt);
        }
        __syncwarp();  // the lane groups leave the queue apart; the barrier wants whole warps
        if (!(ok = team.sync(ctl))) break;

        // termination test (Alg. 1), next threshold: one thread per CTA reads
        // the iteration's counters and shares them through shared memory (a
        // read by every warp of the team would queue hundreds of requests on
        // the same L2 line)
        unsigned* term = fused_term;
        if (threadIdx.x == 0) {
            const unsigned long long gk = tc.ld(&ctl->gk3[set]);
            term[0] = (unsigned)tc.ld(&ctl->goal3[set]);
            term[1] = (unsigned)(gk >> 32);
            term[2] = (unsigned)(gk & 0xffffffffu);
            term[3] = (unsigned)tc.ld(&ctl->new3[set]);
            term[4] = min(tc.ld(&ctl->min_keep3[set]), tc.ld(&ctl->min_new3[set]));
        }
        __syncthreads();
        const int goal = (int)term[0];
        const int kept = (int)term[1], ngrp = (int)term[2];
        const int opened = (int)term[3];
        const unsigned mk = term[4];
        ++it;
        if (goal) { status = GMT_OK; break; }
        if (kept + opened == 0) { status = GMT_NO_PATH; break; }
        nk = kept;
        nn = opened;
        ng_prev = ngrp;
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

    // the copy of the counters in CTA 0 has been read for the last time by
    // every CTA before any of them leaves
    if (SH) team.sync(ctl);

    // ---- result: counters (every commit happened before the last barrier),
    // the returned path
    if (ok) {
        unsigned long long checks = cnt.checks, failed = cnt.failed, computed = cnt.computed,
                           tree = (unsigned long long)cnt.tree + n_tree;
        unsigned long long n_push = cnt.push, n_pull = cnt.pull;
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
    int* const spar = reinterpret_cast<int*>(sbox);
    const bool par_in_smem = ok && status == GMT_OK && (size_t)N * sizeof(int) <= sbox_bytes;
    if (par_in_smem && team.cta() == 0) {  // uniform over CTA 0
        for (int v = threadIdx.x; v < N; v += blockDim.x) spar[v] = ldcg_i(&A.parent[v]);
        __syncthreads();
    }
    if (rank == 0) {
        const int err = tc.ld(&ctl->error);
        ctl->status = err ? err : status;
        ctl->goal_key = tc.ld(&ctl->goal_key);  // the host reads the goal's cost from it
        ctl->iters = it;
        ctl->final_i = (int)i;
        ctl->goal_node = -1;
        ctl->path_len = 0;
        if (ok && status == GMT_OK) {
            const int g = (int)(tc.ld(&ctl->goal_key) & 0xffffffffu);
            ctl->goal_node = g;
            auto parent_of = [&](int v) { return par_in_smem ? spar[v] : ldcg_i(&A.parent[v]); };
            int len = 1, v = g;
            while (v > 0 && len <= N) {
                v = parent_of(v);
                ++len;
            }
            if (v != 0) len = 0;
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

}  // namespace gmtk
