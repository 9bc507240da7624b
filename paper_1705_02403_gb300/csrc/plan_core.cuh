// Team synchronisation primitives and the lazy edge checks shared by the
// wavefront kernels (plan.cu: one query per team; plan_multi.cu: all queries
// of a batch advancing together).
#pragma once

#include <climits>

#include "common.cuh"
#include "internal.h"

namespace gmtk {

constexpr int kDefaultSpinLimit = 1 << 22;

__device__ __forceinline__ int ldcg_i(const int* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned ldcg_u(const unsigned* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg_f(const float* p) { return __ldcg(p); }

// Every team also names its CTAs (cta() in [0, ctas())), so that work can be
// dealt to CTAs round-robin.
struct BlockTeam {
    static constexpr bool kSharedCtl = true;  // the team's counters can live in shared memory
    __device__ __forceinline__ int id() const { return blockIdx.x; }
    __device__ __forceinline__ int cta() const { return 0; }
    __device__ __forceinline__ int ctas() const { return 1; }
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ bool sync(PlanCtl*) const {
        __syncthreads();
        return true;
    }
};

// Sense-reversing barrier over all CTAs of a cooperative grid.  Every poll is
// counted; after spin_limit polls (or once another CTA has reported an error)
// the wait gives up, records GMT_ERR_TIMEOUT and returns false, so the kernel
// ends with an error status instead of hanging.
struct GridTeam {
    static constexpr bool kSharedCtl = false;
    unsigned expected;
    int spin_limit;
    __device__ __forceinline__ int id() const { return 0; }
    __device__ __forceinline__ int cta() const { return blockIdx.x; }
    __device__ __forceinline__ int ctas() const { return gridDim.x; }
    __device__ __forceinline__ int rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ int size() const { return gridDim.x * blockDim.x; }
    __device__ bool sync(PlanCtl* ctl) const {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned gen = ld_acquire(&ctl->bar_gen);
            const unsigned arrived = atom_add_acq_rel(&ctl->bar_count, 1u);
            if (arrived == expected - 1) {
                ctl->bar_count = 0;
                st_release(&ctl->bar_gen, gen + 1);
            } else {
                int spins = 0;
                while (ld_acquire(&ctl->bar_gen) == gen) {
                    if (ld_volatile(&ctl->error) != 0) break;
                    if (++spins > spin_limit) {
                        atomicCAS(&ctl->error, 0, (int)GMT_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        __syncthreads();
        return ld_volatile(&ctl->error) == 0;
    }
};

// All CTAs of one thread-block cluster (up to 16 SMs of a GPC).  The barrier
// is the hardware cluster barrier (arrive.release / wait.acquire at cluster
// scope); it cannot wait forever because every thread of the cluster reaches
// every barrier (all exits from the iteration loop are uniform).
struct ClusterTeam {
    static constexpr bool kSharedCtl = true;
    __device__ __forceinline__ static unsigned cta_rank() {
        unsigned r;
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
        return r;
    }
    __device__ __forceinline__ static unsigned cluster_ctas() {
        unsigned n;
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
        return n;
    }
    __device__ __forceinline__ int id() const { return (int)(blockIdx.x / cluster_ctas()); }
    __device__ __forceinline__ int cta() const { return (int)cta_rank(); }
    __device__ __forceinline__ int ctas() const { return (int)cluster_ctas(); }
    __device__ __forceinline__ int rank() const { return (int)(cta_rank() * blockDim.x + threadIdx.x); }
    __device__ __forceinline__ int size() const { return (int)(cluster_ctas() * blockDim.x); }
    __device__ __forceinline__ bool sync(PlanCtl*) const {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        return true;
    }
};

// ------------------------------------------------------------- lane groups
// A group of W lanes (W = 32: the warp; W = 16: half a warp) working on one
// edge: its lane index, its lanes' mask, and votes whose bit i is lane i of
// the group.  Two groups of one warp may call these at the same time with
// their own masks.
template <int W>
struct LaneGroup {
    static_assert(W == 32 || W == 16 || W == 8, "lane groups of 8, 16 or 32 lanes");
    __device__ __forceinline__ static int base() { return (int)(threadIdx.x & 31) & ~(W - 1); }
    __device__ __forceinline__ static int lane() { return (int)threadIdx.x & (W - 1); }
    __device__ __forceinline__ static unsigned mask() {
        return W == 32 ? 0xffffffffu : ((1u << (W & 31)) - 1u) << base();
    }
    __device__ __forceinline__ static unsigned ballot(bool p) {
        const unsigned b = __ballot_sync(mask(), p);
        return W == 32 ? b : (b >> base()) & ((1u << (W & 31)) - 1u);
    }
    __device__ __forceinline__ static bool any(bool p) { return __any_sync(mask(), p); }
};

// ------------------------------------------------------------ team counters
// The wavefront's team-wide counters (PlanCtl's group, queue and commit
// words): in the control block in global memory (SH = false), or in a copy in
// the shared memory of the team's first CTA (SH = true: a CTA or a cluster),
// reached through the cluster's shared window, where a dependent atomic takes
// about a third of a global one's latency (measured on GB300: 261 against 707
// cycles; a load 219 against 307).  Field addresses are those of the control
// block; `base` maps them into the copy.  The ordering of the memory model
// holds in both: barrier.cluster (or __syncthreads) orders the copy's
// accesses across the team, and the fences of the global path also order the
// queue's global entries against these counters (acquire/release at cluster
// scope covers both state spaces).
template <bool SH>
struct TeamCtl {
    PlanCtl* g;
    unsigned base;  // SH: shared::cluster address of the copy in CTA 0
    template <class T>
    __device__ __forceinline__ unsigned at(const T* f) const {
        return base + (unsigned)((const char*)f - (const char*)g);
    }
    __device__ __forceinline__ int add(int* f, int v) const {
        if (!SH) return atomicAdd(f, v);
        int r;
        asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(r) : "r"(at(f)), "r"(v) : "memory");
        return r;
    }
    __device__ __forceinline__ unsigned add(unsigned* f, unsigned v) const {
        if (!SH) return atomicAdd(f, v);
        unsigned r;
        asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(r) : "r"(at(f)), "r"(v) : "memory");
        return r;
    }
    __device__ __forceinline__ unsigned long long add(unsigned long long* f, unsigned long long v) const {
        if (!SH) return atomicAdd(f, v);
        unsigned long long r;
        asm volatile("atom.shared::cluster.add.u64 %0, [%1], %2;" : "=l"(r) : "r"(at(f)), "l"(v) : "memory");
        return r;
    }
    __device__ __forceinline__ void min(unsigned* f, unsigned v) const {
        if (!SH) { atomicMin(f, v); return; }
        unsigned r;
        asm volatile("atom.shared::cluster.min.u32 %0, [%1], %2;" : "=r"(r) : "r"(at(f)), "r"(v) : "memory");
    }
    // 64-bit minimum: a compare-and-swap loop in the copy (on GB300 the
    // native 64-bit atomic minimum through the cluster's shared window lost
    // updates under contention in a test of 16 CTAs, while 64-bit add and CAS
    // were exact); every failed CAS returns a smaller value, so the loop ends.
    __device__ __forceinline__ void min(unsigned long long* f, unsigned long long v) const {
        if (!SH) { atomicMin(f, v); return; }
        const unsigned a = at(f);
        unsigned long long cur;
        asm volatile("ld.relaxed.cluster.shared::cluster.u64 %0, [%1];" : "=l"(cur) : "r"(a) : "memory");
        while (v < cur) {
            unsigned long long prev;
            asm volatile("atom.shared::cluster.cas.b64 %0, [%1], %2, %3;" : "=l"(prev) : "r"(a), "l"(cur), "l"(v) : "memory");
            if (prev == cur) break;
            cur = prev;
        }
    }
    __device__ __forceinline__ void cas(int* f, int cmp, int v) const {
        if (!SH) { atomicCAS(f, cmp, v); return; }
        int r;
        asm volatile("atom.shared::cluster.cas.b32 %0, [%1], %2, %3;" : "=r"(r) : "r"(at(f)), "r"(cmp), "r"(v) : "memory");
    }
    // relaxed (volatile) load; acquire load at cluster scope
    __device__ __forceinline__ int ld(const int* f) const {
        if (!SH) return ld_volatile(f);
        int r;
        asm volatile("ld.relaxed.cluster.shared::cluster.u32 %0, [%1];" : "=r"(r) : "r"(at(f)) : "memory");
        return r;
    }
    __device__ __forceinline__ unsigned ld(const unsigned* f) const {
        if (!SH) return __ldcg(f);
        unsigned r;
        asm volatile("ld.relaxed.cluster.shared::cluster.u32 %0, [%1];" : "=r"(r) : "r"(at(f)) : "memory");
        return r;
    }
    __device__ __forceinline__ unsigned long long ld(const unsigned long long* f) const {
        if (!SH) return __ldcg(f);
        unsigned long long r;
        asm volatile("ld.relaxed.cluster.shared::cluster.u64 %0, [%1];" : "=l"(r) : "r"(at(f)) : "memory");
        return r;
    }
    __device__ __forceinline__ unsigned ld_acq(const unsigned* f) const {
        if (!SH) return ld_acquire(f);
        unsigned r;
        asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(r) : "r"(at(f)) : "memory");
        return r;
    }
    // plain stores (the writer then passes a team barrier before any reader)
    __device__ __forceinline__ void st(int* f, int v) const {
        if (!SH) { *f = v; return; }
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(at(f)), "r"(v) : "memory");
    }
    __device__ __forceinline__ void st(unsigned* f, unsigned v) const {
        if (!SH) { *f = v; return; }
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(at(f)), "r"(v) : "memory");
    }
    __device__ __forceinline__ void st(unsigned long long* f, unsigned long long v) const {
        if (!SH) { *f = v; return; }
        asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(at(f)), "l"(v) : "memory");
    }
};

// The shared::cluster address of `p` (this CTA's shared memory) in CTA `rank`
// of the cluster (a launch without clusters is a cluster of one CTA).
__device__ __forceinline__ unsigned cluster_map(const void* p, unsigned rank) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// ---------------------------------------------------------------- edge check
// Both checks first keep only the boxes that meet an axis-aligned bound of
// every point the check will evaluate (one box per lane, a lane group's width
// at a time), then test the points against those boxes alone.  The bound is inflated by far
// more than the rounding of the point formulas, so a box that holds one of
// the computed points is never dropped: the verdict equals testing every
// point against every box.

// Does box b meet [lo, hi] (closed intervals on all DP axes)?
template <int DP>
__device__ __forceinline__ bool box_meets(const float* blo, const float* bhi, int b, const float* lo,
                                          const float* hi) {
    bool m = true;
#pragma unroll
    for (int a = 0; a < DP; ++a) m = m && blo[b * DP + a] <= hi[a] && lo[a] <= bhi[b * DP + a];
    return m;
}

// Geometric edge y -> x of length L: m = max(2, ceil(L/spacing) + 1) points
// p_k = y + t_k (x - y), t_k = k/(m-1); collision if one lies in a closed box.
// Without the grid, boxes that do not meet the segment's bounding box (every
// computed p_k lies within a few ulps of it) are set aside W at a time first.
template <int DP, int W = 32>
__device__ __forceinline__ bool segment_free_warp(const float* y, const float* x, float L, float spacing, const float* blo,
                                  const float* bhi, int nbox, const BoxGridArgs& grid) {
    using LG = LaneGroup<W>;
    const int lane = LG::lane();
    int m = (int)ceilf(L / spacing) + 1;
    if (m < 2) m = 2;
    const float denom = (float)(m - 1);
    if (grid.use) {
        for (int k0 = 0; k0 < m; k0 += W) {
            const int k = k0 + lane;
            bool hit = false;
            if (k < m) {
                const float t = (float)k / denom;
                float p[DP];
#pragma unroll
                for (int a = 0; a < DP; ++a) p[a] = y[a] + t * (x[a] - y[a]);
                hit = in_any_box_grid<DP>(p, blo, bhi, grid);
            }
            if (LG::any(hit)) return false;
        }
        return true;
    }
    float lo[DP], hi[DP];
#pragma unroll
    for (int a = 0; a < DP; ++a) {
        const float e = 1e-5f * (fabsf(x[a]) + fabsf(y[a])) + 1e-30f;
        lo[a] = fminf(x[a], y[a]) - e;
        hi[a] = fmaxf(x[a], y[a]) + e;
    }
    for (int b0 = 0; b0 < nbox; b0 += W) {
        const int b = b0 + lane;
        const unsigned near = LG::ballot(b < nbox && box_meets<DP>(blo, bhi, b, lo, hi));
        if (!near) continue;
        for (int k0 = 0; k0 < m; k0 += W) {
            const int k = k0 + lane;
            bool hit = false;
            if (k < m) {
                const float t = (float)k / denom;
                float p[DP];
#pragma unroll
                for (int a = 0; a < DP; ++a) p[a] = y[a] + t * (x[a] - y[a]);
                for (unsigned w = near; w; w &= w - 1) hit = hit || in_box<DP>(p, blo, bhi, b0 + __ffs(w) - 1);
            }
            if (LG::any(hit)) return false;
        }
    }
    return true;
}

// Double-integrator edge: `points` samples of the Hermite trajectory at
// s_k = k/(points-1); collision if one lies in a box or outside the position
// bounds.  Without the grid, the boxes are first filtered against the
// bounding box of the cubic's Bezier control points p0, p0 + tau v0 / 3,
// p1 - tau v1 / 3, p1 (the curve lies in their convex hull), inflated.
template <int W = 32>
__device__ __forceinline__ bool trajectory_free_warp(const float* y, const float* x, float tau, int points, const float* plo,
                                            const float* phi, const float* blo, const float* bhi, int nbox,
                                            const BoxGridArgs& grid) {
    using LG = LaneGroup<W>;
    const int lane = LG::lane();
    const float denom = (float)(points - 1);
    float lo[3], hi[3];
    unsigned near_first = 0;  // boxes 0..W-1, reused by the first chunk of points
    if (!grid.use) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float c1 = y[a] + tau * y[3 + a] / 3.0f, c2 = x[a] - tau * x[3 + a] / 3.0f;
            const float e =
                1e-5f * (fabsf(y[a]) + fabsf(x[a]) + tau * (fabsf(y[3 + a]) + fabsf(x[3 + a]))) + 1e-30f;
            lo[a] = fminf(fminf(y[a], x[a]), fminf(c1, c2)) - e;
            hi[a] = fmaxf(fmaxf(y[a], x[a]), fmaxf(c1, c2)) + e;
        }
        if (nbox > 0) near_first = LG::ballot(lane < nbox && box_meets<3>(blo, bhi, lane, lo, hi));
    }
    for (int k0 = 0; k0 < points; k0 += W) {
        const int k = k0 + lane;
        bool hit = false;
        float p[3];
        if (k < points) {
            const float s = (float)k / denom;
            hermite_point(y, x, tau, s, p);
#pragma unroll
            for (int a = 0; a < 3; ++a) hit = hit || p[a] < plo[a] || p[a] > phi[a];
            if (grid.use && !hit) hit = in_any_box_grid<3>(p, blo, bhi, grid);
        }
        if (!grid.use) {
            for (int b0 = 0; b0 < nbox; b0 += W) {
                const unsigned near =
                    b0 == 0 ? near_first
                            : LG::ballot(b0 + lane < nbox && box_meets<3>(blo, bhi, b0 + lane, lo, hi));
                if (k < points)
                    if (!hit && near) hit = in_near_boxes<3>(p, blo, bhi, b0, near);
            }
        }
        if (LG::any(hit)) return false;
    }
    return true;
}

// Dubins airplane edge y -> x of cost c along its shortest word P:
// m = max(2, ceil(c / spacing) + 1) trajectory points at fractions k / (m - 1);
// a point in a box or outside the position bounds collides.  Every lane walks
// the segment start poses once, then its own points.  Without the box grid,
// boxes are first tested against a bound of the whole trajectory: its planar
// part stays within c/2 of the midpoint of y and x (a point at arc length l is
// within l of y and L - l of x, L <= c), its altitude between the two end
// altitudes.
template <int W = 32>
__device__ __forceinline__ bool dubins_free_warp(const float* y, const float* x, const DubPath& P, float c,
                                                 float spacing, float rho, const float* plo, const float* phi,
                                                 const float* blo, const float* bhi, int nbox,
                                                 const BoxGridArgs& grid) {
    using LG = LaneGroup<W>;
    const int lane = LG::lane();
    if (P.word >= kDubNone) return false;  // no word: never an edge (its cost would be +inf)
    const DubSegs G = dubins_segments(y, P, rho);
    int m = (int)ceilf(c / spacing) + 1;
    if (m < 2) m = 2;
    const float denom = (float)(m - 1);
    float lo[3], hi[3];
    unsigned near_first = 0;
    if (!grid.use) {
        const float e = 1e-3f * c + 1e-5f * (fabsf(y[0]) + fabsf(y[1]) + fabsf(y[2]) + rho) + 1e-30f;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float mid = 0.5f * (y[a] + x[a]);
            lo[a] = mid - 0.5f * c - e;
            hi[a] = mid + 0.5f * c + e;
        }
        lo[2] = fminf(y[2], x[2]) - e;
        hi[2] = fmaxf(y[2], x[2]) + e;
        if (nbox > 0) near_first = LG::ballot(lane < nbox && box_meets<3>(blo, bhi, lane, lo, hi));
    }
    for (int k0 = 0; k0 < m; k0 += W) {
        const int k = k0 + lane;
        bool hit = false;
        float p[3];
        if (k < m) {
            dubins_point(y, x, G, (float)k / denom, p);
#pragma unroll
            for (int a = 0; a < 3; ++a) hit = hit || p[a] < plo[a] || p[a] > phi[a];
            if (grid.use && !hit) hit = in_any_box_grid<3>(p, blo, bhi, grid);
        }
        if (!grid.use) {
            for (int b0 = 0; b0 < nbox; b0 += W) {
                const unsigned near =
                    b0 == 0 ? near_first
                            : LG::ballot(b0 + lane < nbox && box_meets<3>(blo, bhi, b0 + lane, lo, hi));
                if (k < m)
                    if (!hit && near) hit = in_near_boxes<3>(p, blo, bhi, b0, near);
            }
        }
        if (LG::any(hit)) return false;
    }
    return true;
}

// Loads of the wavefront's mutable state (snapshot, lists, control block):
// from L2 (ld.global.cg) when the team spans several SMs, plain loads when a
// single CTA keeps that state in its shared memory (SM = true).
template <bool SM> __device__ __forceinline__ int st_i(const int* p) { if (SM) return *p; return __ldcg(p); }
template <bool SM> __device__ __forceinline__ unsigned st_u(const unsigned* p) { if (SM) return *p; return __ldcg(p); }
template <bool SM> __device__ __forceinline__ float st_f(const float* p) { if (SM) return *p; return __ldcg(p); }
template <bool SM> __device__ __forceinline__ int2 st_i2(const int2* p) { if (SM) return *p; return __ldcg(p); }
template <bool SM> __device__ __forceinline__ unsigned long long st_ull(const unsigned long long* p) {
    if (SM) return *p;
    return __ldcg(p);
}

// Lazy parent (Alg. 1, Sec. III-A), one lane's share of a group of W lanes:
// over the in-row entries r0 + lane, r0 + lane + W, ... the minimum (cost, index) of
// fl(ocost[y] + in_cost[e]) among open y (ocost < +inf); *be = its edge, -1
// if none.  (cost, index) is a total order, so the order of the entries does
// not matter: four chunks of W are taken at a time, their column and cost
// loads issued together, then their snapshot gathers.
template <bool SM, int W = 32>
__device__ __forceinline__ void lane_parent_min(const int* __restrict__ in_col, const float* __restrict__ in_cost,
                                                const float* ocost, int r0, int r1, int lane, float* bc_out,
                                                int* by_out, int* be_out) {
    const float INF = f_inf();
    float bc = INF;
    int by = INT_MAX, be = -1;
    for (int eb = r0; eb < r1; eb += 4 * W) {
        int ys[4];
        float ic[4], oc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = eb + W * u + lane;
            ys[u] = e < r1 ? __ldg(&in_col[e]) : -1;
            ic[u] = e < r1 ? __ldg(&in_cost[e]) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) oc[u] = ys[u] >= 0 ? st_f<SM>(&ocost[ys[u]]) : INF;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (oc[u] < INF) {
                const float c = oc[u] + ic[u];
                if (c < bc || (c == bc && ys[u] < by)) { bc = c; by = ys[u]; be = eb + W * u + lane; }
            }
        }
    }
    *bc_out = bc;
    *by_out = by;
    *be_out = be;
}


// Shared-memory layout of the single-CTA kernel that keeps the wavefront state
// on chip (plan_kernel_smem): region0 (boxes / parent copy), the control
// block, ocost and stamp (N each), the lists.
__host__ __device__ constexpr size_t smem_round16(size_t b) { return (b + 15) / 16 * 16; }
constexpr size_t kSmemCtlBytes = smem_round16(sizeof(PlanCtl));
inline size_t plan_smem_state_bytes(size_t region0, int N) {
    return smem_round16(region0) + kSmemCtlBytes + smem_round16((size_t)8 * N) +
           smem_round16(plan_list_stride((size_t)N) * sizeof(int));
}

}  // namespace gmtk
