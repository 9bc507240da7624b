// Device building blocks of the GB300 GMT* planner: Philox4x32-10, the
// connection costs, point-in-box tests and bounded inter-block waits.
//
// All floating-point decisions use IEEE FP32 with round-to-nearest; the
// library is compiled with -fmad=false -prec-div=true -prec-sqrt=true
// -ftz=false, and every expression below is written in the evaluation order
// the planner's specification fixes (left to right), so results are
// reproducible bit for bit.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dubins.cuh"
#include "gmt.h"
#include "internal.h"

namespace gmtk {

constexpr int kMaxDim = GMT_MAX_DIM;
constexpr int kWarp = 32;

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

// Hardware approximations (a few ulp): used only where a result feeds a
// conservative filter with ample slack, never in a decision the oracle checks.
__device__ __forceinline__ float approx_sqrt(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float approx_rcp(float x) {
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  A round maps the counter
// (c0, c1, c2, c3) under key (k0, k1) to
//   (hi(B c2) ^ c1 ^ k0, lo(B c2), hi(A c0) ^ c3 ^ k1, lo(A c0)),
// A = 0xD2511F53, B = 0xCD9E8D57; the key advances by (0x9E3779B9, 0xBB67AE85)
// after every round.  Ten rounds.
// ---------------------------------------------------------------------------
struct Ctr4 { uint32_t x, y, z, w; };

__device__ __forceinline__ Ctr4 philox4x32_10(Ctr4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hiA = __umulhi(0xD2511F53u, c.x), loA = 0xD2511F53u * c.x;
        const uint32_t hiB = __umulhi(0xCD9E8D57u, c.z), loB = 0xCD9E8D57u * c.z;
        c = Ctr4{hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Top 24 bits of a word scaled by 2^-24: exact, in [0, 1).
__device__ __forceinline__ float unit_float(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

// ---------------------------------------------------------------------------
// Obstacles: closed axis-aligned boxes, lo[b*DP + a] <= p[a] <= hi[b*DP + a].
// ---------------------------------------------------------------------------
template <int DP>
__device__ __forceinline__ bool in_box(const float* p, const float* lo, const float* hi, int b) {
    bool inside = true;
#pragma unroll
    for (int a = 0; a < DP; ++a) inside = inside && (lo[b * DP + a] <= p[a]) && (p[a] <= hi[b * DP + a]);
    return inside;
}

// Does p lie in one of the boxes b0 + i, i a set bit of `near`?  Four boxes per
// step with every comparison evaluated (no short circuit), so their loads
// issue together; the answer is that of testing them one by one.
template <int DP>
__device__ __forceinline__ bool in_near_boxes(const float* p, const float* lo, const float* hi, int b0,
                                              unsigned near) {
    bool hit = false;
    for (unsigned w = near; w;) {
        const int first = b0 + __ffs(w) - 1;
        bool h = false;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool valid = w != 0u;
            const int b = valid ? b0 + __ffs(w) - 1 : first;
            w &= w - 1u;
            bool inside = valid;
#pragma unroll
            for (int a = 0; a < DP; ++a) inside = inside & (lo[b * DP + a] <= p[a]) & (p[a] <= hi[b * DP + a]);
            h = h | inside;
        }
        hit = hit | h;
    }
    return hit;
}

template <int DP>
__device__ __forceinline__ bool in_any_box(const float* p, const float* lo, const float* hi, int nbox) {
    for (int b = 0; b < nbox; ++b)
        if (in_box<DP>(p, lo, hi, b)) return true;
    return false;
}

// Grid cell of coordinate x on grid axis a, clamped to the grid.
__device__ __forceinline__ int box_grid_cell(const BoxGridArgs& g, float x, int a) {
    const int k = (int)floorf((x - g.lo[a]) * g.inv_h[a]);
    return min(max(k, 0), g.g - 1);
}

// Does point p lie in a box?  With the grid, only the boxes listed in p's
// cell and the big boxes can hold it; each is tested exactly.  One thread.
template <int DP>
__device__ __forceinline__ bool in_any_box_grid(const float* p, const float* blo, const float* bhi,
                                                const BoxGridArgs& grid) {
    const int c = box_grid_cell(grid, p[1], 1) * grid.g + box_grid_cell(grid, p[0], 0);
    const int e = __ldg(&grid.start[c + 1]);
    for (int t = __ldg(&grid.start[c]); t < e; ++t)
        if (in_box<DP>(p, blo, bhi, __ldg(&grid.list[t]))) return true;
    const int nb = __ldg(grid.nbig);
    for (int t = 0; t < nb; ++t)
        if (in_box<DP>(p, blo, bhi, __ldg(&grid.big[t]))) return true;
    return false;
}

// Is p in any box: through the grid when the caller built one, else by
// scanning every box.
template <int DP>
__device__ __forceinline__ bool point_in_boxes(const float* p, const gmtk::BoxArgs& boxes,
                                               const gmtk::BoxGridArgs& grid) {
    return grid.use ? in_any_box_grid<DP>(p, boxes.lo, boxes.hi, grid) : in_any_box<DP>(p, boxes.lo, boxes.hi, boxes.count);
}

// ---------------------------------------------------------------------------
// Euclidean cost: sqrt of sum_a (to_a - from_a)^2 accumulated in axis order.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ float sq_dist(const float* from, const float* to) {
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float t = to[a] - from[a];
        s = s + t * t;
    }
    return s;
}

// ---------------------------------------------------------------------------
// Double integrator (3 axes, state [p v]): for fixed arrival time tau the
// minimum-effort cost is J(tau) = tau + a/tau - b/tau^2 + c/tau^3 with
//   a = 4(|v0|^2 + v0.v1 + |v1|^2), b = 12 dp.(v0+v1), c = 12 |dp|^2;
// the optimal tau is the smallest positive root of
//   q(tau) = tau^4 - a tau^2 + 2b tau - 3c = ((tau tau - a) tau + 2b) tau - 3c,
// bracketed on tau_k = r (k/32), k = 1..32 (first k with q >= 0, none -> no
// edge since J >= tau) and refined by 24 halvings (q(mid) < 0 -> lo = mid).
// J is evaluated as ((c/tau - b)/tau + a)/tau + tau.
// ---------------------------------------------------------------------------
struct DICoef { float a, b, c, b2, c3; };

__device__ __forceinline__ DICoef di_coef(const float* s0, const float* s1) {
    float n00 = 0.0f, n01 = 0.0f, n11 = 0.0f, bs = 0.0f, cs = 0.0f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float p0 = s0[ax], v0 = s0[3 + ax], p1 = s1[ax], v1 = s1[3 + ax];
        const float dp = p1 - p0;
        n00 = n00 + v0 * v0;
        n01 = n01 + v0 * v1;
        n11 = n11 + v1 * v1;
        bs = bs + dp * (v0 + v1);
        cs = cs + dp * dp;
    }
    DICoef k;
    k.a = 4.0f * ((n00 + n01) + n11);
    k.b = 12.0f * bs;
    k.c = 12.0f * cs;
    k.b2 = 2.0f * k.b;
    k.c3 = 3.0f * k.c;
    return k;
}

__device__ __forceinline__ float di_q(const DICoef& k, float t) { return ((t * t - k.a) * t + k.b2) * t - k.c3; }

constexpr int kDIGrid = 32;
constexpr int kDIBisect = 24;

// Arrival time tau* (or +inf when no root lies in (0, r]).
__device__ __forceinline__ float di_tau(const DICoef& k, float r) {
    float lo = 0.0f, hi = f_inf();
    for (int g = 1; g <= kDIGrid; ++g) {
        const float tg = r * ((float)g / (float)kDIGrid);
        if (di_q(k, tg) >= 0.0f) { hi = tg; break; }
        lo = tg;
    }
    if (hi == f_inf()) return hi;
    for (int s = 0; s < kDIBisect; ++s) {
        const float mid = lo + (hi - lo) * 0.5f;
        if (di_q(k, mid) < 0.0f) lo = mid; else hi = mid;
    }
    return hi;
}

// Two arrival times at once, each bit-identical to di_tau: the same grid
// points and the same halvings, with the two searches interleaved so that
// their dependent chains overlap.  The grid is scanned two points per step
// (the first point with q >= 0 wins, as in the one-point scan).
__device__ __forceinline__ void di_tau2(const DICoef& k0, const DICoef& k1, float r, float& t0, float& t1) {
    static_assert(kDIGrid % 2 == 0, "two grid points per step");
    // g0, g1: the first grid index with q >= 0 (0 while none is found)
    int g0 = 0, g1 = 0;
    for (int g = 1; g <= kDIGrid; g += 2) {
        const float ta = r * ((float)g / (float)kDIGrid), tb = r * ((float)(g + 1) / (float)kDIGrid);
        const bool a0 = di_q(k0, ta) >= 0.0f, b0 = di_q(k0, tb) >= 0.0f;
        const bool a1 = di_q(k1, ta) >= 0.0f, b1 = di_q(k1, tb) >= 0.0f;
        if (g0 == 0) g0 = a0 ? g : b0 ? g + 1 : 0;
        if (g1 == 0) g1 = a1 ? g : b1 ? g + 1 : 0;
        if (g0 != 0 && g1 != 0) break;
    }
    // the bracket [tau_{g-1}, tau_g] (tau_0 = 0); an edge without a root in
    // (0, r] takes lo = hi = 0, so its halvings stay finite, and +inf
    float lo0 = g0 > 1 ? r * ((float)(g0 - 1) / (float)kDIGrid) : 0.0f;
    float hi0 = g0 > 0 ? r * ((float)g0 / (float)kDIGrid) : 0.0f;
    float lo1 = g1 > 1 ? r * ((float)(g1 - 1) / (float)kDIGrid) : 0.0f;
    float hi1 = g1 > 0 ? r * ((float)g1 / (float)kDIGrid) : 0.0f;
    for (int s = 0; s < kDIBisect; ++s) {
        const float m0 = lo0 + (hi0 - lo0) * 0.5f, m1 = lo1 + (hi1 - lo1) * 0.5f;
        const bool n0 = di_q(k0, m0) < 0.0f, n1 = di_q(k1, m1) < 0.0f;
        lo0 = n0 ? m0 : lo0;
        hi0 = n0 ? hi0 : m0;
        lo1 = n1 ? m1 : lo1;
        hi1 = n1 ? hi1 : m1;
    }
    t0 = g0 > 0 ? hi0 : f_inf();
    t1 = g1 > 0 ? hi1 : f_inf();
}

__device__ __forceinline__ float di_J(const DICoef& k, float t) { return ((k.c / t - k.b) / t + k.a) / t + t; }

// Cost from state s0 to state s1 (+inf when no root lies in (0, r]).
__device__ __forceinline__ float di_cost(const float* s0, const float* s1, float r) {
    const DICoef k = di_coef(s0, s1);
    const float t = di_tau(k, r);
    if (t == f_inf()) return t;
    return di_J(k, t);
}

// Conservative rejection of pairs that cannot have J < r (never rejects an
// edge; the exact procedure decides the rest).  With s = v0 + v1, dv = v1 - v0
// the cost is exactly
//   J(tau) = tau + |dv|^2 / tau + 3 |2 dp - s tau|^2 / tau^3.
// For tau in (0, r], |2 dp - s tau| >= D, the distance from the point 2 dp to
// the segment {s t : 0 <= t <= r}, so J(tau) >= f(tau) = tau + A/tau + B/tau^3
// with A = |dv|^2, B = 3 D^2.  f is convex with f'(t) = 0 at
// t^2 = (A + sqrt(A^2 + 12 B)) / 2, so min over (0, r] of f is f(min(t, r)).
// A pair whose bound reaches r (inflated by 1% to absorb FP32 rounding, far
// above the few-ulp error of either side) cannot be an edge.  The bound only
// filters (the exact procedure decides every pair it keeps), so it may use the
// fast reciprocal and square-root approximations: their few-ulp error is far
// inside the 1% slack.
__device__ __forceinline__ bool di_may_connect(const float* s0, const float* s1, float r) {
    const float rr = r * 1.01f;
    float A = 0.0f, qs = 0.0f, ss = 0.0f, q[3], sv[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float dv = s1[3 + ax] - s0[3 + ax];
        A = A + dv * dv;
        q[ax] = 2.0f * (s1[ax] - s0[ax]);
        sv[ax] = s0[3 + ax] + s1[3 + ax];
        qs = qs + q[ax] * sv[ax];
        ss = ss + sv[ax] * sv[ax];
    }
    if (4.0f * A >= rr * rr) return false;  // f >= 2 sqrt(A)
    float t = ss > 0.0f ? __fdividef(qs, ss) : 0.0f;
    t = fminf(fmaxf(t, 0.0f), rr);
    float D2 = 0.0f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float e = q[ax] - t * sv[ax];
        D2 = D2 + e * e;
    }
    const float B = 3.0f * D2;
    float tau = approx_sqrt(0.5f * (A + approx_sqrt(A * A + 12.0f * B)));
    tau = fminf(tau, rr);
    if (!(tau > 0.0f)) return true;
    const float inv = approx_rcp(tau);
    const float f = tau + A * inv + B * (inv * inv * inv);
    return f < rr;
}

// Second filter stage, for the pairs di_may_connect keeps.  With R = 1.01 r,
// q(tau) = tau^3 (J(tau) - R) = tau^4 - R tau^3 + a tau^2 - b tau + c.  The exact
// procedure only reports an edge when J(tau*) < r at a root tau* in (0, r], and
// J(tau*) >= min of J over (0, r], so an edge needs q <= 0 somewhere in (0, r].
// On each quarter [lo, lo + h] of [0, r] the Bernstein coefficients of q
// (degree 4) bound q from below; if every coefficient of every quarter exceeds
// T = 1e-4 S (S = |c| + |b| r + a r^2 + R r^3 + r^4 bounds every term's size, and
// the FP32 rounding of these few operations stays below 1e-5 S), q > 0 on
// (0, r] and the pair cannot be an edge.  The 1% slack covers the rounding of
// the exact procedure's J, as for the bound above.
__device__ __forceinline__ bool di_bern_may_connect(const float* s0, const float* s1, float r) {
    const DICoef k = di_coef(s0, s1);
    const float R = r * 1.01f;
    const float a = k.a, b = k.b, c = k.c;
    const float r2 = r * r;
    const float S = fabsf(c) + fabsf(b) * r + fabsf(a) * r2 + R * r2 * r + r2 * r2;
    const float T = 1e-4f * S;
    const float h = 0.25f * r;
    const float h2 = h * h;
    const float d4 = h2 * h2;
#pragma unroll
    for (int qtr = 0; qtr < 4; ++qtr) {
        const float lo = (float)qtr * h;
        // Taylor coefficients of q at lo times powers of h: q(lo + h s) = sum d_k s^k
        const float d0 = (((lo - R) * lo + a) * lo - b) * lo + c;
        const float d1 = (((4.0f * lo - 3.0f * R) * lo + 2.0f * a) * lo - b) * h;
        const float d2 = ((6.0f * lo - 3.0f * R) * lo + a) * h2;
        const float d3 = (4.0f * lo - R) * h2 * h;
        // Bernstein coefficients: beta_i = sum_{k <= i} C(i,k) / C(4,k) d_k
        const float b1 = d0 + 0.25f * d1;
        const float b2 = (d0 + 0.5f * d1) + d2 * (1.0f / 6.0f);
        const float b3 = ((d0 + 0.75f * d1) + 0.5f * d2) + 0.25f * d3;
        const float b4 = (((d0 + d1) + d2) + d3) + d4;
        if (!(d0 > T && b1 > T && b2 > T && b3 > T && b4 > T)) return true;
    }
    return false;
}

// Position of the minimum-effort trajectory (cubic Hermite curve) at s in [0,1]:
//   p = ((h00 p0 + (h10 tau) v0) + h01 p1) + (h11 tau) v1,
//   h00 = (2 s^3 - 3 s^2) + 1, h10 = (s^3 - 2 s^2) + s, h01 = 3 s^2 - 2 s^3,
//   h11 = s^3 - s^2, s^2 = s s, s^3 = s^2 s.
__device__ __forceinline__ void hermite_point(const float* s0, const float* s1, float tau, float s, float* p) {
    const float s2 = s * s;
    const float s3 = s2 * s;
    const float h00 = (2.0f * s3 - 3.0f * s2) + 1.0f;
    const float h10 = (s3 - 2.0f * s2) + s;
    const float h01 = 3.0f * s2 - 2.0f * s3;
    const float h11 = s3 - s2;
    const float h10t = h10 * tau, h11t = h11 * tau;
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = ((h00 * s0[a] + h10t * s0[3 + a]) + h01 * s1[a]) + h11t * s1[3 + a];
}

// ---------------------------------------------------------------------------
// Memory-ordered global accesses for inter-block synchronisation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ void st_volatile_i(int* p, int v) { *(volatile int*)p = v; }

// Warp-aggregated append: every lane with `want` gets a distinct slot of
// list[*count], one atomic per warp.  Returns the slot (or -1).
__device__ __forceinline__ int warp_append_slot(bool want, int* count) {
    const unsigned mask = __ballot_sync(0xffffffffu, want);
    if (mask == 0) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    return want ? base + __popc(mask & ((1u << lane) - 1u)) : -1;
}

__device__ __forceinline__ unsigned float_key(float c) { return __float_as_uint(c); }  // c >= 0

}  // namespace gmtk
