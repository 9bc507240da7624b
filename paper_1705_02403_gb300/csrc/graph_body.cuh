// Device-function bodies of the SampleFree and neighbour-graph kernels,
// shared by the single-problem kernels (graph.cu) and the batched ones
// (batch.cu), so both run the same arithmetic.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace gmtk {


// ------------------------------------------------------------------ sampling
__device__ __forceinline__ bool in_goal_ball(const float* x, int gd, const float* c, float rho) {
    float s = 0.0f;
    for (int a = 0; a < gd; ++a) {
        const float t = x[a] - c[a];
        s = s + t * t;
    }
    return s <= rho * rho;
}

template <int D, int DP>
__device__ __forceinline__ void sample_node(const SpaceArgs& s, const BoxArgs& boxes, const BoxGridArgs& grid,
                                            float* __restrict__ X, uint8_t* __restrict__ is_goal,
                                            int* __restrict__ flags, int k) {
    if (k >= s.n_sampled) return;
    float x[D];
    if (k == 0) {
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            x[a] = s.x0[a];
            ok = ok && s.lo[a] <= x[a] && x[a] <= s.hi[a];
        }
        if (!ok || point_in_boxes<DP>(x, boxes, grid)) atomicOr(flags, kSampleBadInit);
    } else {
        bool ok = false;
        for (int t = 0; t < s.max_attempts && !ok; ++t) {
            uint32_t w[((D + 3) / 4) * 4];
#pragma unroll
            for (int blk = 0; blk < (D + 3) / 4; ++blk) {
                const Ctr4 c = philox4x32_10(Ctr4{(uint32_t)k, (uint32_t)t, s.stream, (uint32_t)blk}, s.key0, s.key1);
                w[4 * blk + 0] = c.x; w[4 * blk + 1] = c.y; w[4 * blk + 2] = c.z; w[4 * blk + 3] = c.w;
            }
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float u = unit_float(w[a]);
                float l = s.lo[a], h = s.hi[a];
                if (k == 1 && a < s.gd) { l = s.gc[a] - s.grho; h = s.gc[a] + s.grho; }
                x[a] = l + u * (h - l);
            }
            if (k == 1) {
                bool inb = true;
#pragma unroll
                for (int a = 0; a < D; ++a) inb = inb && s.lo[a] <= x[a] && x[a] <= s.hi[a];
                if (!inb || !in_goal_ball(x, s.gd, s.gc, s.grho)) continue;
            }
            if (point_in_boxes<DP>(x, boxes, grid)) continue;
            ok = true;
        }
        if (!ok) atomicOr(flags, kSampleExhausted);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) X[(size_t)a * s.pitch + k] = x[a];
    is_goal[k] = in_goal_ball(x, s.gd, s.gc, s.grho) ? 1 : 0;
}

// Attempt t of SampleFree for node k >= 1 (the draws of sample_node): x
// receives the attempt's state; returns whether it is accepted (node 1: in
// the goal region and in X; every node: outside every box).  FLAT: the box
// test visits every box with no early exit and no short-circuit (the same
// answer, no divergence inside it).
template <int D, int DP, bool FLAT>
__device__ __forceinline__ bool sample_attempt(const SpaceArgs& s, const BoxArgs& boxes, const BoxGridArgs& grid,
                                               int k, int t, float* x) {
    uint32_t w[((D + 3) / 4) * 4];
#pragma unroll
    for (int blk = 0; blk < (D + 3) / 4; ++blk) {
        const Ctr4 c = philox4x32_10(Ctr4{(uint32_t)k, (uint32_t)t, s.stream, (uint32_t)blk}, s.key0, s.key1);
        w[4 * blk + 0] = c.x; w[4 * blk + 1] = c.y; w[4 * blk + 2] = c.z; w[4 * blk + 3] = c.w;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float u = unit_float(w[a]);
        float l = s.lo[a], h = s.hi[a];
        if (k == 1 && a < s.gd) { l = s.gc[a] - s.grho; h = s.gc[a] + s.grho; }
        x[a] = l + u * (h - l);
    }
    if (k == 1) {
        bool inb = true;
#pragma unroll
        for (int a = 0; a < D; ++a) inb = inb && s.lo[a] <= x[a] && x[a] <= s.hi[a];
        if (!inb || !in_goal_ball(x, s.gd, s.gc, s.grho)) return false;
    }
    if (FLAT && !grid.use) {
        bool hit = false;
        for (int b = 0; b < boxes.count; ++b) {
            bool in = true;
#pragma unroll
            for (int a = 0; a < DP; ++a)
                in = in & (boxes.lo[b * DP + a] <= x[a]) & (x[a] <= boxes.hi[b * DP + a]);
            hit = hit | in;
        }
        return !hit;
    }
    return !point_in_boxes<DP>(x, boxes, grid);
}

// The same sample drawn by a group of G consecutive lanes (G divides 32):
// every lane of the group computes the same attempt (the same Philox words),
// and the box tests of an attempt are dealt round-robin over the group's
// lanes and ORed with shuffles, so an attempt's chain is about nbox / G box
// tests long instead of nbox.  Lane `sub` = 0 writes the result.  The
// accepted attempt, and so the sample, is the one sample_node takes.
template <int D, int DP, int G>
__device__ __forceinline__ bool point_in_boxes_group(const float* p, const BoxArgs& boxes, const BoxGridArgs& grid,
                                                     int sub, unsigned gmask) {
    bool hit = false;
    if (grid.use) {
        const int c = box_grid_cell(grid, p[1], 1) * grid.g + box_grid_cell(grid, p[0], 0);
        const int e = __ldg(&grid.start[c + 1]);
        for (int t = __ldg(&grid.start[c]) + sub; t < e; t += G) hit |= in_box<DP>(p, boxes.lo, boxes.hi, __ldg(&grid.list[t]));
        const int nb = __ldg(grid.nbig);
        for (int t = sub; t < nb; t += G) hit |= in_box<DP>(p, boxes.lo, boxes.hi, __ldg(&grid.big[t]));
    } else {
        for (int b = sub; b < boxes.count; b += G) hit |= in_box<DP>(p, boxes.lo, boxes.hi, b);
    }
#pragma unroll
    for (int off = 1; off < G; off <<= 1) hit |= __shfl_xor_sync(gmask, hit ? 1 : 0, off) != 0;
    return hit;
}

// SampleFree for node k on a group of Q * P lanes of one warp: P attempts at
// once (attempts t0 .. t0 + P - 1), each on Q lanes that share out its box
// tests.  The node takes the first accepted attempt in attempt order, the one
// the sequential rejection loop would take.
template <int D, int DP, int Q, int P>
__device__ __forceinline__ void sample_node_group(const SpaceArgs& s, const BoxArgs& boxes, const BoxGridArgs& grid,
                                                  float* __restrict__ X, uint8_t* __restrict__ is_goal,
                                                  int* __restrict__ flags, int k) {
    constexpr int G = Q * P;
    static_assert(32 % G == 0, "a group lies within one warp");
    if (k >= s.n_sampled) return;  // uniform over the group
    const int lane = threadIdx.x & 31, sub = lane % G, q = sub % Q, first = lane - sub;
    const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << first;
    const unsigned qmask = ((1u << Q) - 1u) << (lane - q);
    float x[D] = {};
    if (k == 0) {
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            x[a] = s.x0[a];
            ok = ok && s.lo[a] <= x[a] && x[a] <= s.hi[a];
        }
        const bool hit = point_in_boxes_group<D, DP, G>(x, boxes, grid, sub, gmask);
        if (sub == 0 && (!ok || hit)) atomicOr(flags, kSampleBadInit);
    } else {
        bool found = false;
        for (int t0 = 0; t0 < s.max_attempts && !found; t0 += P) {  // uniform over the group
            const int t = t0 + sub / Q;
            bool acc = false;
            if (t < s.max_attempts) {  // uniform over the attempt's Q lanes
                uint32_t w[((D + 3) / 4) * 4];
#pragma unroll
                for (int blk = 0; blk < (D + 3) / 4; ++blk) {
                    const Ctr4 c =
                        philox4x32_10(Ctr4{(uint32_t)k, (uint32_t)t, s.stream, (uint32_t)blk}, s.key0, s.key1);
                    w[4 * blk + 0] = c.x; w[4 * blk + 1] = c.y; w[4 * blk + 2] = c.z; w[4 * blk + 3] = c.w;
                }
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const float u = unit_float(w[a]);
                    float l = s.lo[a], h = s.hi[a];
                    if (k == 1 && a < s.gd) { l = s.gc[a] - s.grho; h = s.gc[a] + s.grho; }
                    x[a] = l + u * (h - l);
                }
                acc = true;
                if (k == 1) {
#pragma unroll
                    for (int a = 0; a < D; ++a) acc = acc && s.lo[a] <= x[a] && x[a] <= s.hi[a];
                    acc = acc && in_goal_ball(x, s.gd, s.gc, s.grho);
                }
                if (acc) acc = !point_in_boxes_group<D, DP, Q>(x, boxes, grid, q, qmask);
            }
            // the first accepted attempt of the round (one vote per attempt)
            const unsigned m = (__ballot_sync(gmask, acc && q == 0) >> first) & (G == 32 ? 0xffffffffu : ((1u << G) - 1u));
            if (m) {
                found = true;
                const int src = first + __ffs(m) - 1;
#pragma unroll
                for (int a = 0; a < D; ++a) x[a] = __shfl_sync(gmask, x[a], src);
            }
        }
        if (!found && sub == 0) atomicOr(flags, kSampleExhausted);
    }
    if (sub != 0) return;
#pragma unroll
    for (int a = 0; a < D; ++a) X[(size_t)a * s.pitch + k] = x[a];
    is_goal[k] = in_goal_ball(x, s.gd, s.gc, s.grho) ? 1 : 0;
}

// ------------------------------------------------------------ Halton
// Radical inverse of k in base p, exactly: the digits of k reversed (R) over
// p^m (m digits), rounded to double and then to float (R, p^m < 2^35).
__host__ __device__ __forceinline__ float halton_unit(uint32_t k, uint32_t p) {
    unsigned long long R = 0, P = 1;
    while (k > 0) {
        R = R * p + k % p;
        P *= p;
        k /= p;
    }
    return (float)((double)R / (double)P);
}

__host__ __device__ __forceinline__ uint32_t halton_prime(int a) {
    const uint32_t primes[10] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29};
    return primes[a];
}

constexpr int kHaltonThreads = 512;

// Halton point k mapped onto X, and whether it is free (outside every box).
template <int D, int DP>
__device__ __forceinline__ bool halton_free_point(const SpaceArgs& s, const BoxArgs& boxes, const BoxGridArgs& grid,
                                                  long long k, float* x) {
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = s.lo[a] + halton_unit((uint32_t)k, halton_prime(a)) * (s.hi[a] - s.lo[a]);
    return !point_in_boxes<DP>(x, boxes, grid);
}

// Nodes 0 and 1 of a Halton SampleFree, run by a whole block: node 0 =
// x_init (and its checks); node 1 = the first goal-mapped point (smallest k)
// in X, in the goal ball and outside the boxes.  Writes their goal flags.
template <int D, int DP>
__device__ void halton_head_block(const SpaceArgs& s, const BoxArgs& boxes, const BoxGridArgs& grid,
                                  float* __restrict__ X, uint8_t* __restrict__ is_goal, int* __restrict__ flags) {
    __shared__ int s_best;
    const int tid = threadIdx.x;
    if (tid == 0) sample_node<D, DP>(s, boxes, grid, X, is_goal, flags, 0);  // x_init, its checks and goal flag
    // node 1
    if (tid == 0) s_best = INT_MAX;
    __syncthreads();
    for (long long base = 1; base <= s.halton_cap; base += blockDim.x) {
        const long long k = base + tid;
        if (k <= s.halton_cap) {
            float x[D];
            bool ok = true;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float u = halton_unit((uint32_t)k, halton_prime(a));
                float l = s.lo[a], h = s.hi[a];
                if (a < s.gd) { l = s.gc[a] - s.grho; h = s.gc[a] + s.grho; }
                x[a] = l + u * (h - l);
                ok = ok && s.lo[a] <= x[a] && x[a] <= s.hi[a];
            }
            if (ok && in_goal_ball(x, s.gd, s.gc, s.grho) && !point_in_boxes<DP>(x, boxes, grid))
                atomicMin(&s_best, (int)k);
        }
        __syncthreads();
        const bool found = s_best != INT_MAX;
        __syncthreads();
        if (found) break;
    }
    if (tid == 0) {
        if (s_best == INT_MAX) {
            atomicOr(flags, kSampleExhausted);
        } else {
            float x[D];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float u = halton_unit((uint32_t)s_best, halton_prime(a));
                float l = s.lo[a], h = s.hi[a];
                if (a < s.gd) { l = s.gc[a] - s.grho; h = s.gc[a] + s.grho; }
                x[a] = l + u * (h - l);
                X[(size_t)a * s.pitch + 1] = x[a];
            }
            is_goal[1] = in_goal_ball(x, s.gd, s.gc, s.grho) ? 1 : 0;
        }
    }
}

// Halton SampleFree of one graph, run by a whole block of kHaltonThreads:
// nodes 0 and 1 as halton_head_block; nodes 2..n_sampled-1 = the free points
// in the order of k (block-wide prefix sums keep that order).
template <int D, int DP>
__device__ void halton_sample_block(const SpaceArgs& s, const BoxArgs& boxes, const BoxGridArgs& grid,
                                    float* __restrict__ X, uint8_t* __restrict__ is_goal, int* __restrict__ flags) {
    __shared__ int s_warp[kHaltonThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int N = s.n_sampled;
    halton_head_block<D, DP>(s, boxes, grid, X, is_goal, flags);
    // nodes 2..N-1
    int got = 0;
    for (long long base = 1; got < N - 2; base += blockDim.x) {
        if (base > s.halton_cap) {
            if (tid == 0) atomicOr(flags, kSampleExhausted);
            break;
        }
        const long long k = base + tid;
        float x[D];
        bool ok = false;
        if (k <= s.halton_cap) ok = halton_free_point<D, DP>(s, boxes, grid, k, x);
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < nwarps; ++w) {
            const int c = s_warp[w];
            before += w < warp ? c : 0;
            total += c;
        }
        const int rank = before + __popc(m & ((1u << lane) - 1u));
        if (ok && got + rank < N - 2) {
#pragma unroll
            for (int a = 0; a < D; ++a) X[(size_t)a * s.pitch + 2 + got + rank] = x[a];
        }
        got += total;
        __syncthreads();
    }
    __syncthreads();
    for (int v = tid; v < N; v += blockDim.x) {
        float x[D];
#pragma unroll
        for (int a = 0; a < D; ++a) x[a] = X[(size_t)a * s.pitch + v];
        is_goal[v] = in_goal_ball(x, s.gd, s.gc, s.grho) ? 1 : 0;
    }
}

// Appended sample k (one thread): copy, goal flag, validity (inside X, outside
// every box).
template <int D, int DP>
__device__ __forceinline__ void append_node(const SpaceArgs& s, const BoxArgs& boxes, const float* __restrict__ src,
                                            int src_pitch, int first, float* __restrict__ X,
                                            uint8_t* __restrict__ is_goal, int* __restrict__ flags, int k) {
    float x[D];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x[a] = src[(size_t)a * src_pitch + k];
        ok = ok && s.lo[a] <= x[a] && x[a] <= s.hi[a];
        X[(size_t)a * s.pitch + first + k] = x[a];
    }
    if (!ok || in_any_box<DP>(x, boxes.lo, boxes.hi, boxes.count)) atomicOr(flags, kSampleBadAppend);
    is_goal[first + k] = in_goal_ball(x, s.gd, s.gc, s.grho) ? 1 : 0;
}

// ------------------------------------------------------------- pair filter
constexpr int kMaskRows = 256;     // rows (threads) per block
constexpr int kMaskWords = 8;      // 32-column words per block (256 columns staged in shared memory)

template <int KIND, int D>
__device__ __forceinline__ bool connects(const SpaceArgs& s, const float* from, const float* to) {
    if (KIND == GMT_COST_EUCLID) return sq_dist<D>(from, to) < s.r2_threshold;
    if (KIND == GMT_COST_DUBINS) return dubins_near(from, to, s.r) && dubins_cost(from, to, s.rho) < s.r;
    if (!di_may_connect(from, to, s.r)) return false;
    return di_cost(from, to, s.r) < s.r;
}

template <int KIND, int D>
__device__ __forceinline__ float edge_cost(const SpaceArgs& s, const float* from, const float* to) {
    if (KIND == GMT_COST_EUCLID) return __fsqrt_rn(sq_dist<D>(from, to));
    if (KIND == GMT_COST_DUBINS) return dubins_cost(from, to, s.rho);
    return di_cost(from, to, s.r);
}

// Packed FP32 pairs (two IEEE round-to-nearest operations per instruction,
// each lane of the pair rounded on its own: the same bits as two scalar ops).
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// di_may_connect for two pairs at once (s0a -> s1a and s0b -> s1b): the same
// operations in the same order, the additions and multiplications packed two
// to an instruction, so each verdict is the scalar function's.
__device__ __forceinline__ void di_may_connect_x2(const float* s0a, const float* s1a, const float* s0b,
                                                  const float* s1b, float r, bool& pass_a, bool& pass_b) {
    const float rr = r * 1.01f;
    const unsigned long long two = f2_pack(2.0f, 2.0f);
    unsigned long long A = f2_pack(0.0f, 0.0f), qs = A, ss = A, q[3], sv[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const unsigned long long v0 = f2_pack(s0a[3 + ax], s0b[3 + ax]), v1 = f2_pack(s1a[3 + ax], s1b[3 + ax]);
        const unsigned long long dv = f2_sub(v1, v0);
        A = f2_add(A, f2_mul(dv, dv));
        q[ax] = f2_mul(two, f2_sub(f2_pack(s1a[ax], s1b[ax]), f2_pack(s0a[ax], s0b[ax])));
        sv[ax] = f2_add(v0, v1);
        qs = f2_add(qs, f2_mul(q[ax], sv[ax]));
        ss = f2_add(ss, f2_mul(sv[ax], sv[ax]));
    }
    float Aa, Ab, qsa, qsb, ssa, ssb;
    f2_unpack(A, Aa, Ab);
    f2_unpack(qs, qsa, qsb);
    f2_unpack(ss, ssa, ssb);
    float ta = ssa > 0.0f ? __fdividef(qsa, ssa) : 0.0f, tb = ssb > 0.0f ? __fdividef(qsb, ssb) : 0.0f;
    ta = fminf(fmaxf(ta, 0.0f), rr);
    tb = fminf(fmaxf(tb, 0.0f), rr);
    const unsigned long long t = f2_pack(ta, tb);
    unsigned long long D2 = f2_pack(0.0f, 0.0f);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const unsigned long long e = f2_sub(q[ax], f2_mul(t, sv[ax]));
        D2 = f2_add(D2, f2_mul(e, e));
    }
    const unsigned long long B = f2_mul(f2_pack(3.0f, 3.0f), D2);
    const unsigned long long disc = f2_add(f2_mul(A, A), f2_mul(f2_pack(12.0f, 12.0f), B));
    float da, db;
    f2_unpack(disc, da, db);
    const unsigned long long h = f2_mul(f2_pack(0.5f, 0.5f), f2_add(A, f2_pack(approx_sqrt(da), approx_sqrt(db))));
    float ha, hb;
    f2_unpack(h, ha, hb);
    const float taua = fminf(approx_sqrt(ha), rr), taub = fminf(approx_sqrt(hb), rr);
    const unsigned long long tau = f2_pack(taua, taub), inv = f2_pack(approx_rcp(taua), approx_rcp(taub));
    const unsigned long long f =
        f2_add(f2_add(tau, f2_mul(A, inv)), f2_mul(B, f2_mul(f2_mul(inv, inv), inv)));
    float fa, fb;
    f2_unpack(f, fa, fb);
    const float rr2 = rr * rr;
    pass_a = !(4.0f * Aa >= rr2) && (!(taua > 0.0f) || fa < rr);
    pass_b = !(4.0f * Ab >= rr2) && (!(taub > 0.0f) || fb < rr);
}

// Euclidean graphs of 2 to 4 dimensions: columns are staged in pairs (float4
// (x_j, x_j+1, y_j, y_j+1), then (z_j, z_j+1, w_j, w_j+1)), and each lane
// tests its row against two columns per step with packed FP32 arithmetic:
// t = x_j - x_i, then d2 = t_0^2 + t_1^2 + ... in axis order, which is the
// expression of sq_dist (0 + t_0^2 = t_0^2 exactly), so the bits are the same.
// Columns past the last node hold +inf (an infinite distance: no edge), so
// the inner loop tests no bounds; the diagonal pair i = j is cleared once per
// word.  tile_cnt (or NULL): receives the row's edge count in this tile's
// columns at [by * pitch + i], for the tiled fill.
template <int D>
__device__ __forceinline__ void mask_tile_euclid4(const SpaceArgs& s, const float* __restrict__ X,
                                                  uint32_t* __restrict__ mask, int* __restrict__ out_count, int bx,
                                                  int by, int* __restrict__ tile_cnt) {
    static_assert(D >= 2 && D <= 4, "two to four axes in two float4s per column pair");
    constexpr int kPairs = kMaskWords * 16;
    __shared__ float4 tab[kPairs];                  // axes 0 and 1
    __shared__ float4 tcd[D > 2 ? kPairs : 1];      // axes 2 and 3
    const int i = bx * kMaskRows + threadIdx.x;
    const int w0 = by * kMaskWords;
    const int j0 = w0 * 32;
    const float INF = f_inf();
    for (int idx = threadIdx.x; idx < kPairs; idx += kMaskRows) {
        const int ja = j0 + 2 * idx, jb = ja + 1;
        float c[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            c[0][a] = ja < s.N ? X[(size_t)a * s.pitch + ja] : INF;
            c[1][a] = jb < s.N ? X[(size_t)a * s.pitch + jb] : INF;
        }
        tab[idx] = make_float4(c[0][0], c[1][0], c[0][1], c[1][1]);
        if (D > 2) tcd[idx] = make_float4(c[0][2], c[1][2], c[0][3], c[1][3]);
    }
    __syncthreads();
    if (i >= s.N) return;
    unsigned long long xi2[4];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float v = X[(size_t)a * s.pitch + i];
        xi2[a] = f2_pack(v, v);
    }
    const int W = (s.N + 31) / 32;
    const float thr = s.r2_threshold;
    int cnt = 0;
    for (int ww = 0; ww < kMaskWords; ++ww) {
        const int w = w0 + ww;
        if (w >= W) break;
        uint32_t bits = 0;
#pragma unroll
        for (int b = 0; b < 32; b += 2) {
            const float4 q = tab[ww * 16 + (b >> 1)];
            const unsigned long long t0 = f2_sub(f2_pack(q.x, q.y), xi2[0]);
            const unsigned long long t1 = f2_sub(f2_pack(q.z, q.w), xi2[1]);
            unsigned long long d2 = f2_add(f2_mul(t0, t0), f2_mul(t1, t1));
            if (D > 2) {
                const float4 r = tcd[ww * 16 + (b >> 1)];
                const unsigned long long t2 = f2_sub(f2_pack(r.x, r.y), xi2[2]);
                d2 = f2_add(d2, f2_mul(t2, t2));
                if (D > 3) {
                    const unsigned long long t3 = f2_sub(f2_pack(r.z, r.w), xi2[3]);
                    d2 = f2_add(d2, f2_mul(t3, t3));
                }
            }
            float da, db;
            f2_unpack(d2, da, db);
            bits |= (da < thr ? 1u : 0u) << b;
            bits |= (db < thr ? 1u : 0u) << (b + 1);
        }
        if ((i >> 5) == w) bits &= ~(1u << (i & 31));  // no self-loop
        mask[(size_t)w * s.pitch + i] = bits;
        cnt += __popc(bits);
    }
    if (cnt) atomicAdd(&out_count[i], cnt);
    if (tile_cnt) tile_cnt[(size_t)by * s.pitch + i] = cnt;
}

// Tiled fill of a Euclidean graph of 2 to 4 dimensions (after
// mask_tile_euclid4 with tile_cnt and the row scan): tile_prefix_row turns a
// row's per-tile counts into exclusive prefixes (nb tiles of kMaskWords words
// each); then fill_tile_euclid, one block per mask tile with the tile's
// columns staged in shared memory, writes each row's columns of the tile, in
// ascending order, from row[i] + prefix, with cost sqrt(d2) of the same
// expression as edge_cost (so the same bits), and no gather of the samples
// per edge.  Each lane loads its row's words; the warp then deals all its
// rows' columns of the tile to its lanes in order, so no lane idles while
// another walks a long row, and a row's columns go to consecutive lanes.
__device__ __forceinline__ void tile_prefix_row(int* __restrict__ tile_cnt, int pitch, int nb, int i) {
    constexpr int kChunk = 16;  // loads issued together, then the chunk's prefixes stored
    int acc = 0;
    for (int b0 = 0; b0 < nb; b0 += kChunk) {
        int c[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) c[u] = b0 + u < nb ? tile_cnt[(size_t)(b0 + u) * pitch + i] : 0;
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
            if (b0 + u < nb) tile_cnt[(size_t)(b0 + u) * pitch + i] = acc;
            acc += c[u];
        }
    }
}

// Position of the m-th (from 0) set bit of x (x has more than m set bits):
// the largest p with fewer than m + 1 set bits below it, by binary search.
__device__ __forceinline__ int select_bit(uint32_t x, int m) {
    int p = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (__popc(x & ((1u << (p + step)) - 1u)) <= m) p += step;
    return p;
}

template <int D>
__device__ __forceinline__ void fill_tile_euclid(const SpaceArgs& s, const float* __restrict__ X,
                                                 const uint32_t* __restrict__ mask, const int* __restrict__ row,
                                                 const int* __restrict__ tile_pre, int* __restrict__ col,
                                                 float* __restrict__ cost, int bx, int by) {
    static_assert(D >= 2 && D <= 4, "float4 columns");
    constexpr int kWarps = kMaskRows / 32;
    __shared__ float4 tile[kMaskWords * 32];
    __shared__ uint32_t swords[kWarps][32][kMaskWords];  // each row's words of the tile
    __shared__ int sex[kWarps][33];                       // exclusive prefix of the rows' column counts
    __shared__ int sbase[kWarps][32];                     // each row's first position for the tile
    __shared__ float4 sxi[kWarps][32];                    // each row's coordinates
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = bx * kMaskRows + threadIdx.x;
    const int w0 = by * kMaskWords;
    const int j0 = w0 * 32;
    for (int idx = threadIdx.x; idx < kMaskWords * 32; idx += kMaskRows) {
        const int j = j0 + idx;
        float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < D; ++a) c[a] = j < s.N ? X[(size_t)a * s.pitch + j] : 0.0f;
        tile[idx] = make_float4(c[0], c[1], c[2], c[3]);
    }
    // each lane loads its row's words of the tile (coalesced over the rows)
    const bool row_ok = i < s.N;
    const int W = (s.N + 31) / 32;
    int cnt = 0;
#pragma unroll
    for (int ww = 0; ww < kMaskWords; ++ww) {
        const uint32_t w = row_ok && w0 + ww < W ? mask[(size_t)(w0 + ww) * s.pitch + i] : 0u;
        swords[warp][lane][ww] = w;
        cnt += __popc(w);
    }
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < D; ++a) c[a] = row_ok ? X[(size_t)a * s.pitch + i] : 0.0f;
    sxi[warp][lane] = make_float4(c[0], c[1], c[2], c[3]);
    sbase[warp][lane] = cnt > 0 ? row[i] + tile_pre[(size_t)by * s.pitch + i] : 0;
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    sex[warp][lane] = incl - cnt;
    if (lane == 31) sex[warp][32] = incl;
    __syncthreads();  // the staged columns; the warp's row tables
    // the warp's columns in (row, word, bit) order, dealt to its lanes: entry
    // e of row r goes to position sbase[r] + (e - sex[r]), so each row's
    // columns come out ascending and consecutive lanes write consecutive
    // positions of a row
    const int total = sex[warp][32];
    for (int e = lane; e < total; e += 32) {
        int r = 0;  // the row: the last one whose prefix is <= e
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (sex[warp][r + step] <= e) r += step;
        int m = e - sex[warp][r], k = 0;
        uint32_t wk = swords[warp][r][0];
        for (int ww = 0; ww < kMaskWords; ++ww) {
            wk = swords[warp][r][ww];
            const int cw = __popc(wk);
            if (m < cw) { k = ww; break; }
            m -= cw;
        }
        const int jt = k * 32 + select_bit(wk, m);
        const float4 q = tile[jt], p = sxi[warp][r];
        const float xj[4] = {q.x, q.y, q.z, q.w}, xr[4] = {p.x, p.y, p.z, p.w};
        float d2 = 0.0f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const float tt = xj[a] - xr[a];
            d2 = d2 + tt * tt;
        }
        const int pos = sbase[warp][r] + (e - sex[warp][r]);
        col[pos] = j0 + jt;
        cost[pos] = __fsqrt_rn(d2);
    }
}

// One block of kMaskRows threads: rows bx*kMaskRows.., words by*kMaskWords..
template <int KIND, int D>
__device__ __forceinline__ void mask_tile(const SpaceArgs& s, const float* __restrict__ X,
                                          uint32_t* __restrict__ mask, int* __restrict__ out_count, int bx,
                                          int by, int* __restrict__ tile_cnt = nullptr) {
    if constexpr (KIND == GMT_COST_EUCLID && D >= 2 && D <= 4) {
        mask_tile_euclid4<D>(s, X, mask, out_count, bx, by, tile_cnt);
        return;
    }
    __shared__ float tile[D][kMaskWords * 32];
    const int i = bx * kMaskRows + threadIdx.x;
    const int w0 = by * kMaskWords;
    const int j0 = w0 * 32;
    for (int idx = threadIdx.x; idx < kMaskWords * 32; idx += kMaskRows) {
        const int j = j0 + idx;
#pragma unroll
        for (int a = 0; a < D; ++a) tile[a][idx] = j < s.N ? X[(size_t)a * s.pitch + j] : 0.0f;
    }
    __syncthreads();
    if (i >= s.N) return;
    float xi[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xi[a] = X[(size_t)a * s.pitch + i];
    const int W = (s.N + 31) / 32;
    int cnt = 0;
    for (int ww = 0; ww < kMaskWords; ++ww) {
        const int w = w0 + ww;
        if (w >= W) break;
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int j = w * 32 + b;
            if (j >= s.N || j == i) continue;
            float xj[D];
#pragma unroll
            for (int a = 0; a < D; ++a) xj[a] = tile[a][ww * 32 + b];
            if (connects<KIND, D>(s, xi, xj)) bits |= 1u << b;
        }
        mask[(size_t)w * s.pitch + i] = bits;
        cnt += __popc(bits);
    }
    if (cnt) atomicAdd(&out_count[i], cnt);
}

// Double-integrator pair filter.  The exact test (root bracketing + 24
// halvings, ~400 FP32 operations) is needed only for the ~9% of pairs that
// pass the conservative lower bound, so each warp first evaluates the bound
// for its 32 rows against every staged column and queues the survivors
// (row lane, column) in shared memory; whenever 32 are queued, the warp runs
// the exact test on all of them at once (every lane busy), ORing the verdicts
// into per-row words kept in shared memory.  Rows are the lanes' own rows, so
// a queued pair fetches its row state from the owning lane with a shuffle.
#ifndef GMT_DI_ROWS
#define GMT_DI_ROWS 128
#endif
#ifndef GMT_DI_WORDS
#define GMT_DI_WORDS 1
#endif
constexpr int kDIRows = GMT_DI_ROWS;    // rows (threads) per block
constexpr int kDIWords = GMT_DI_WORDS;  // 32-column words per block (staged columns); 1 measured fastest

// One block of kDIRows threads: rows bx*kDIRows.., words by*kDIWords..
// maskT, in_count (may be NULL): also write the tile's words of the transposed
// (in-neighbour) matrix and count the in-edges, as transpose_task would.
// elist (may be NULL): every edge found is also listed as (row, column, cost
// bits, arrival-time bits) at a slot taken from *elist_n (slots at or past
// elist_cap are counted but not written), so the CSR fill need not solve for
// the arrival time again.
__device__ __forceinline__ void mask_di_tile(const SpaceArgs& s, const float* __restrict__ X,
                                             uint32_t* __restrict__ mask, int* __restrict__ out_count, int bx,
                                             int by, uint32_t* __restrict__ maskT = nullptr,
                                             int* __restrict__ in_count = nullptr, int4* __restrict__ elist = nullptr,
                                             int* __restrict__ elist_n = nullptr, int elist_cap = 0) {
    static_assert(kDIWords == 1, "the first stage keeps a lane's columns in one 32-bit word");
    __shared__ __align__(16) float tile[6][kDIWords * 32];  // float2 reads of column pairs
    __shared__ uint32_t words[kDIRows / 32][kDIWords][32];
    __shared__ uint16_t queue0[kDIRows / 32][32 * 32];  // every pair of the warp's tile may pass the first test
    __shared__ uint16_t queue[kDIRows / 32][3][96];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = bx * kDIRows + threadIdx.x;
    const int w0 = by * kDIWords;
    const int j0 = w0 * 32;
    for (int idx = threadIdx.x; idx < kDIWords * 32; idx += kDIRows) {
        const int j = j0 + idx;
#pragma unroll
        for (int a = 0; a < 6; ++a) tile[a][idx] = j < s.N ? X[(size_t)a * s.pitch + j] : 0.0f;
    }
#pragma unroll
    for (int ww = 0; ww < kDIWords; ++ww) words[warp][ww][lane] = 0u;
    __syncthreads();
    const bool row_ok = i < s.N;
    float xi[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) xi[a] = row_ok ? X[(size_t)a * s.pitch + i] : 0.0f;

    // Four tests of increasing cost and strength: the velocity test of
    // di_may_connect alone (every pair), di_may_connect, di_bern_may_connect,
    // and the exact cost.  Pairs that pass a test wait in that stage's queue;
    // 32 at a time (one per lane) they take the next test, so every lane stays
    // busy although fewer pairs reach each stage.  An entry is
    // (row lane << 8) | column.
    const float rr = s.r * 1.01f;
    int qn0 = 0, qn1 = 0, qn2 = 0;
    auto state = [&](int e, float* a_, float* b_) {
        const int src = e >> 8, jt = e & 255;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            a_[a] = __shfl_sync(0xffffffffu, xi[a], src);
            b_[a] = tile[a][jt];
        }
    };
    // appends the lanes that pass to queue k; returns the new length
    auto enqueue = [&](int k, bool pass, int e, int qn) {
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        if (pass) queue[warp][k][qn + __popc(m & ((1u << lane) - 1u))] = (uint16_t)e;
        __syncwarp();
        return qn + __popc(m);
    };
    // drops the first c (<= 32) of the qn (<= 96) entries of queue k
    auto shift = [&](int k, int qn, int c) {
        __syncwarp();
        const uint16_t m0 = lane + c < qn ? queue[warp][k][lane + c] : (uint16_t)0;
        const uint16_t m1 = lane + 32 + c < qn ? queue[warp][k][lane + 32 + c] : (uint16_t)0;
        __syncwarp();
        if (lane < qn - c) queue[warp][k][lane] = m0;
        if (lane + 32 < qn - c) queue[warp][k][lane + 32] = m1;
        __syncwarp();
        return qn - c;
    };
    auto drain2 = [&](int count) {  // exact test (the steps of di_cost) on queue 2's first count entries
        const int e = lane < count ? queue[warp][2][lane] : 0;
        float a_[6], b_[6];
        state(e, a_, b_);
        const int src = e >> 8, jt = e & 255;
        float J = f_inf(), t = f_inf();
        if (lane < count) {
            const DICoef k = di_coef(a_, b_);
            t = di_tau(k, s.r);
            if (t != f_inf()) J = di_J(k, t);
        }
        const bool edge = J < s.r;
        if (edge) atomicOr(&words[warp][jt >> 5][src], 1u << (jt & 31));
        if (elist) {
            const unsigned m = __ballot_sync(0xffffffffu, edge);
            if (m) {
                int slot = 0;
                if (lane == 0) slot = atomicAdd(elist_n, __popc(m));
                slot = __shfl_sync(0xffffffffu, slot, 0) + __popc(m & ((1u << lane) - 1u));
                if (edge && slot < elist_cap)
                    elist[slot] = make_int4(bx * kDIRows + warp * 32 + src, j0 + jt, __float_as_int(J),
                                            __float_as_int(t));
            }
        }
    };
    auto drain1 = [&](int count) {  // second bound on queue 1's first count entries, into queue 2
        const int e = lane < count ? queue[warp][1][lane] : 0;
        float a_[6], b_[6];
        state(e, a_, b_);
        qn2 = enqueue(2, lane < count && di_bern_may_connect(a_, b_, s.r), e, qn2);
    };
    // first bound on queue0[from, from + count) (count <= 64), into queue 1:
    // each lane takes two entries, evaluated together with packed arithmetic
    auto drain0 = [&](int from, int count) {
        const int ea = lane < count ? queue0[warp][from + lane] : 0;
        const int eb = lane + 32 < count ? queue0[warp][from + 32 + lane] : 0;
        float a0[6], b0[6], a1[6], b1[6];
        state(ea, a0, b0);
        state(eb, a1, b1);
        bool pa, pb;
        di_may_connect_x2(a0, b0, a1, b1, s.r, pa, pb);
        qn1 = enqueue(1, lane < count && pa, ea, qn1);
        qn1 = enqueue(1, lane + 32 < count && pb, eb, qn1);
    };

    const int jend = min(kDIWords * 32, s.N - j0);
    // velocity test for the lane's row against every staged column, one bit
    // per column (J >= tau + |v1 - v0|^2 / tau >= 2 |v1 - v0|); the passing
    // pairs are then queued all at once, so the per-pair cost of the test is
    // its arithmetic and one bit, with no warp vote per column
    uint32_t pm = 0;
    if (row_ok) {
        const float rr2 = rr * rr;
        // two columns per step with packed arithmetic (the staged tile holds 32
        // columns, zero past the last node; bits from jend on are cleared)
        unsigned long long xv2[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) xv2[a] = f2_pack(xi[3 + a], xi[3 + a]);
#pragma unroll 4
        for (int jt = 0; jt < jend; jt += 2) {
            unsigned long long A = f2_pack(0.0f, 0.0f);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float2 c = *reinterpret_cast<const float2*>(&tile[3 + a][jt]);
                const unsigned long long dv = f2_sub(f2_pack(c.x, c.y), xv2[a]);
                A = f2_add(A, f2_mul(dv, dv));
            }
            float A0, A1;
            f2_unpack(A, A0, A1);
            pm |= ((4.0f * A0 < rr2 ? 1u : 0u) | (4.0f * A1 < rr2 ? 2u : 0u)) << jt;
        }
        if (jend < 32) pm &= (1u << jend) - 1u;
        if (i >= j0 && i < j0 + jend) pm &= ~(1u << (i - j0));  // no self pair
    }
    {
        const int np = __popc(pm);
        int incl = np;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        qn0 = __shfl_sync(0xffffffffu, incl, 31);
        int pos = incl - np;
        for (uint32_t m = pm; m; m &= m - 1) queue0[warp][pos++] = (uint16_t)((lane << 8) | (__ffs(m) - 1));
        __syncwarp();
    }
    // The stages as one loop with a single call site each (the instruction
    // cache then holds all of them): a stage runs only when the next one has
    // fewer than 32 entries, so queue 1 holds at most 31 + 64 entries and
    // queue 2 at most 31 + 32; once queue 0 is used up, what is left in
    // queues 1 and 2 is drained.  Every condition is uniform over the warp.
    int from = 0;
#pragma unroll 1
    for (;;) {
        const bool rest = from >= qn0;
        if (qn2 >= 32 || (rest && qn1 == 0 && qn2 > 0)) {
            const int c = min(32, qn2);
            drain2(c);
            qn2 = shift(2, qn2, c);
        } else if (qn1 >= 32 || (rest && qn1 > 0)) {
            const int c = min(32, qn1);
            drain1(c);
            qn1 = shift(1, qn1, c);
        } else if (!rest) {
            drain0(from, min(64, qn0 - from));
            from += 64;
        } else {
            break;
        }
    }
    __syncwarp();
    const int W = (s.N + 31) / 32;
    if (maskT) {
        // transposed: for column j0 + jt, the bits of the warp's 32 rows form
        // word (row chunk, j0 + jt) of the in-neighbour matrix
        const int chunk = (bx * kDIRows) / 32 + warp;
        const uint32_t mine = row_ok ? words[warp][0][lane] : 0u;
        if (chunk < W) {  // uniform over the warp
            uint32_t tw = 0;  // lane jt keeps column j0 + jt's word
#pragma unroll
            for (int jt = 0; jt < 32; ++jt) {
                const uint32_t t = __ballot_sync(0xffffffffu, (mine >> jt) & 1u);
                if (lane == jt) tw = t;
            }
            if (j0 + lane < s.N) {  // one coalesced store and one atomic per lane
                maskT[(size_t)chunk * s.pitch + j0 + lane] = tw;
                if (tw) atomicAdd(&in_count[j0 + lane], __popc(tw));
            }
        }
    }
    if (!row_ok) return;
    int cnt = 0;
#pragma unroll
    for (int ww = 0; ww < kDIWords; ++ww) {
        const int w = w0 + ww;
        if (w >= W) break;
        const uint32_t bits = words[warp][ww][lane];
        mask[(size_t)w * s.pitch + i] = bits;
        cnt += __popc(bits);
    }
    if (cnt) atomicAdd(&out_count[i], cnt);
}

// Dubins airplane pair filter: the 3D-distance prefilter for every pair, then
// the shortest-word cost for the ~3% that pass, 32 at a time from a per-warp
// queue (entry (row lane << 8) | column) so that every lane computes one.
constexpr int kDubRows = 128;  // rows (threads) per block
constexpr int kDubWords = 1;   // 32-column words per block

// maskT, in_count (may be NULL): also write the tile's words of the transposed
// (in-neighbour) matrix and count the in-edges, as transpose_task would.
// elist, epath (may be NULL): every edge is also listed as (row, column, cost
// bits, 0) with its shortest word (t, p, q, word bits) at the same slot of
// epath, slots taken from *elist_n (those at or past elist_cap are counted but
// not written), so the CSR fill need not solve for the word again.
__device__ __forceinline__ void mask_dubins_tile(const SpaceArgs& s, const float* __restrict__ X,
                                                 uint32_t* __restrict__ mask, int* __restrict__ out_count, int bx,
                                                 int by, uint32_t* __restrict__ maskT = nullptr,
                                                 int* __restrict__ in_count = nullptr,
                                                 int4* __restrict__ elist = nullptr,
                                                 float4* __restrict__ epath = nullptr,
                                                 int* __restrict__ elist_n = nullptr, int elist_cap = 0) {
    static_assert(kDubWords == 1, "the prefilter keeps a lane's columns in one 32-bit word");
    __shared__ float tile[4][kDubWords * 32];
    __shared__ uint32_t words[kDubRows / 32][kDubWords][32];
    __shared__ uint16_t queue[kDubRows / 32][32 * 32];  // every pair of the warp's tile may pass the prefilter
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = bx * kDubRows + threadIdx.x;
    const int j0 = by * kDubWords * 32;
    for (int idx = threadIdx.x; idx < kDubWords * 32; idx += kDubRows) {
        const int j = j0 + idx;
#pragma unroll
        for (int a = 0; a < 4; ++a) tile[a][idx] = j < s.N ? X[(size_t)a * s.pitch + j] : 0.0f;
    }
#pragma unroll
    for (int ww = 0; ww < kDubWords; ++ww) words[warp][ww][lane] = 0u;
    __syncthreads();
    const bool row_ok = i < s.N;
    float xi[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) xi[a] = row_ok ? X[(size_t)a * s.pitch + i] : 0.0f;
    // prefilter of the lane's row against every staged column, one bit per
    // column; the passing pairs are then queued all at once and their costs
    // computed 32 at a time (one per lane)
    const int jend = min(kDubWords * 32, s.N - j0);
    uint32_t pm = 0;
    if (row_ok) {
        for (int jt = 0; jt < jend; ++jt) {
            float b_[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) b_[a] = tile[a][jt];
            pm |= (dubins_near(xi, b_, s.r) ? 1u : 0u) << jt;
        }
        if (i >= j0 && i < j0 + jend) pm &= ~(1u << (i - j0));  // no self pair
    }
    int qn;
    {
        const int np = __popc(pm);
        int incl = np;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        qn = __shfl_sync(0xffffffffu, incl, 31);
        int pos = incl - np;
        for (uint32_t m = pm; m; m &= m - 1) queue[warp][pos++] = (uint16_t)((lane << 8) | (__ffs(m) - 1));
        __syncwarp();
    }
    for (int from = 0; from < qn; from += 32) {
        const int count = min(32, qn - from);
        const int e = lane < count ? queue[warp][from + lane] : 0;
        const int src = e >> 8, jt = e & 255;
        float a_[4], b_[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            a_[a] = __shfl_sync(0xffffffffu, xi[a], src);
            b_[a] = tile[a][jt];
        }
        // the steps of dubins_cost
        const DubPath P = dubins_path(a_, b_, s.rho);
        const float c = dubins_length(P, a_, b_);
        const bool edge = lane < count && c < s.r;
        if (edge) atomicOr(&words[warp][jt >> 5][src], 1u << (jt & 31));
        if (elist) {
            const unsigned m = __ballot_sync(0xffffffffu, edge);
            if (m) {
                int slot = 0;
                if (lane == 0) slot = atomicAdd(elist_n, __popc(m));
                slot = __shfl_sync(0xffffffffu, slot, 0) + __popc(m & ((1u << lane) - 1u));
                if (edge && slot < elist_cap) {
                    elist[slot] = make_int4(bx * kDubRows + warp * 32 + src, j0 + jt, __float_as_int(c), 0);
                    epath[slot] = make_float4(P.t, P.p, P.q, __int_as_float(P.word));
                }
            }
        }
    }
    __syncwarp();
    const int W = (s.N + 31) / 32;
    if (maskT) {
        // transposed: for column j0 + jt, the bits of the warp's 32 rows form
        // word (row chunk, j0 + jt) of the in-neighbour matrix
        const int chunk = (bx * kDubRows) / 32 + warp;
        const uint32_t mine = row_ok ? words[warp][0][lane] : 0u;
        if (chunk < W) {  // uniform over the warp
            uint32_t tw = 0;  // lane jt keeps column j0 + jt's word
#pragma unroll
            for (int jt = 0; jt < 32; ++jt) {
                const uint32_t t = __ballot_sync(0xffffffffu, (mine >> jt) & 1u);
                if (lane == jt) tw = t;
            }
            if (j0 + lane < s.N) {  // one coalesced store and one atomic per lane
                maskT[(size_t)chunk * s.pitch + j0 + lane] = tw;
                if (tw) atomicAdd(&in_count[j0 + lane], __popc(tw));
            }
        }
    }
    if (!row_ok) return;
    int cnt = 0;
#pragma unroll
    for (int ww = 0; ww < kDubWords; ++ww) {
        const int w = by * kDubWords + ww;
        if (w >= W) break;
        const uint32_t bits = words[warp][ww][lane];
        mask[(size_t)w * s.pitch + i] = bits;
        cnt += __popc(bits);
    }
    if (cnt) atomicAdd(&out_count[i], cnt);
}

// Word prefixes of a word-major bit matrix (word w of row i at w * pitch + i):
// pre[w * pitch + i] = the set bits of row i's words 0 .. w-1.  One block of
// 1024 threads takes 32 rows (rows0 ..): lane = row, and warp k the k-th
// run of ceil(W / 32) words, so every load is one row-contiguous line.  Each
// warp sums its run, the runs' totals meet in shared memory, and each warp then
// writes its run's prefixes from the sum of the runs before it.
__device__ __forceinline__ void word_prefix_block(const uint32_t* __restrict__ M, int* __restrict__ pre, int N,
                                                  int pitch, int row0) {
    __shared__ int run_total[32][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = (N + 31) / 32, seg = (W + 31) / 32;
    const int i = row0 + lane;
    const int wa = min(W, warp * seg), wb = min(W, wa + seg);
    const bool row_ok = i < N;
    int sum = 0;
    for (int w0 = wa; w0 < wb; w0 += 8) {
        uint32_t b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) b[k] = row_ok && w0 + k < wb ? __ldcg(&M[(size_t)(w0 + k) * pitch + i]) : 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += __popc(b[k]);
    }
    run_total[warp][lane] = sum;
    __syncthreads();
    int run = 0;
    for (int k = 0; k < warp; ++k) run += run_total[k][lane];
    for (int w0 = wa; w0 < wb; w0 += 8) {
        uint32_t b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) b[k] = row_ok && w0 + k < wb ? __ldcg(&M[(size_t)(w0 + k) * pitch + i]) : 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (row_ok && w0 + k < wb) pre[(size_t)(w0 + k) * pitch + i] = run;
            run += __popc(b[k]);
        }
    }
}

// An edge (i, j) listed by a directed pair filter (with its cost bits and, for
// the double integrator, its arrival-time bits; for the Dubins airplane its
// shortest word in `path`), written to both CSRs at its rank: in the out-row
// of i after row[i] + pre[w][i] + the bits of word w = j / 32 below j, in the
// in-row of j the same in the transposed matrix.  The ranks are those the
// row-by-row fill gives, so the CSRs are the same arrays.
template <int KIND>
__device__ __forceinline__ void place_listed_edge(int pitch, int4 q, const float4* path, const FillDir& out,
                                                  const FillDir& in, const int* __restrict__ pre_out,
                                                  const int* __restrict__ pre_in) {
    const int i = q.x, j = q.y;
    const size_t oi = (size_t)(j >> 5) * pitch + i, ij = (size_t)(i >> 5) * pitch + j;
    const int po =
        __ldg(&out.row[i]) + __ldg(&pre_out[oi]) + __popc(__ldg(&out.mask[oi]) & ((1u << (j & 31)) - 1u));
    const int pi = __ldg(&in.row[j]) + __ldg(&pre_in[ij]) + __popc(__ldg(&in.mask[ij]) & ((1u << (i & 31)) - 1u));
    const float c = __int_as_float(q.z);
    out.col[po] = j;
    out.cost[po] = c;
    in.col[pi] = i;
    in.cost[pi] = c;
    if (KIND == GMT_COST_DI) {
        out.tau[po] = __int_as_float(q.w);
        in.tau[pi] = __int_as_float(q.w);
    } else {
        reinterpret_cast<float4*>(in.path)[pi] = *path;
    }
}

// maskT[u][j] bit l = mask[j/32][32u + l] bit (j%32): the in-neighbour rows.
// One warp: the 32x32 bit block `task` = (u, w).
__device__ __forceinline__ void transpose_task(int N, int pitch, const uint32_t* __restrict__ mask,
                                               uint32_t* __restrict__ maskT, int* __restrict__ in_count,
                                               long long task) {
    const int W = (N + 31) / 32;
    const int lane = threadIdx.x & 31;
    if (task >= (long long)W * W) return;
    const int u = (int)(task / W), w = (int)(task % W);
    const int i = 32 * u + lane;
    const uint32_t word = i < N ? mask[(size_t)w * pitch + i] : 0u;
    uint32_t mine = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const uint32_t t = __ballot_sync(0xffffffffu, (word >> b) & 1u);
        if (lane == b) mine = t;
    }
    const int j = 32 * w + lane;
    if (j < N) {
        maskT[(size_t)u * pitch + j] = mine;
        if (mine) atomicAdd(&in_count[j], __popc(mine));
    }
}

// Exclusive prefix sum: row[v] = sum_{u < v} count[u], row[N] = total (also
// returned to every thread).  One block of 1024 threads.
__device__ __forceinline__ int scan_rows(const int* __restrict__ count, int* __restrict__ row, int N) {
    __shared__ int warp_sum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < N; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < N ? count[i] : 0;
        int x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int t = warp_sum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, off);
                if (lane >= off) t += y;
            }
            warp_sum[lane] = t;
        }
        __syncthreads();
        if (i < N) row[i] = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + x - v;
        carry += warp_sum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) row[N] = carry;
    return carry;
}

// Fill: the CSR columns and costs from the bit matrix.  A warp reads a row's
// words 32 at a time (one per lane), prefix-sums the lanes' bit counts and
// writes the columns, in ascending order, to its list in shared memory; the
// listed edges are then evaluated.  Out-rows compute c(v, j), in-rows c(j, v),
// with the same formulas on the same states, so an edge's cost (and arrival
// time, or shortest word) is the same bits in both CSRs and the two
// directions need not wait for each other.
constexpr int kFillWarps = 8;
constexpr int kFillList = 1024;  // column list per warp (a 32-word chunk holds at most 1024)

// The edge between row node v (state xv) and column j, written at CSR position e.
template <int KIND, int D, bool INCOMING>
__device__ __forceinline__ void fill_edge(const SpaceArgs& s, const float* __restrict__ X, const float* xv, int j,
                                          int e, int* __restrict__ col, float* __restrict__ cost,
                                          float* __restrict__ tau, float* __restrict__ path) {
    float xj[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xj[a] = X[(size_t)a * s.pitch + j];
    const float* from = INCOMING ? xj : xv;
    const float* to = INCOMING ? xv : xj;
    float c;
    if (KIND == GMT_COST_DUBINS) {
        const DubPath P = dubins_path(from, to, s.rho);
        c = dubins_length(P, from, to);
        if (path) reinterpret_cast<float4*>(path)[e] = make_float4(P.t, P.p, P.q, __int_as_float(P.word));
    } else if (KIND == GMT_COST_DI) {
        const DICoef k = di_coef(from, to);
        const float t = di_tau(k, s.r);
        c = di_J(k, t);
        tau[e] = t;
    } else {
        c = edge_cost<KIND, D>(s, from, to);
    }
    col[e] = j;
    cost[e] = c;
}

// Two double-integrator edges at once, their root searches interleaved (the
// second is skipped at the stores when !two).
template <int D, bool INCOMING>
__device__ __forceinline__ void fill_edge_di2(const SpaceArgs& s, const float* __restrict__ X, const float* xv0,
                                              int j0, int e0, const float* xv1, int j1, int e1, bool two,
                                              int* __restrict__ col, float* __restrict__ cost,
                                              float* __restrict__ tau) {
    float x0[D], x1[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x0[a] = X[(size_t)a * s.pitch + j0];
        x1[a] = X[(size_t)a * s.pitch + j1];
    }
    const DICoef k0 = INCOMING ? di_coef(x0, xv0) : di_coef(xv0, x0);
    const DICoef k1 = INCOMING ? di_coef(x1, xv1) : di_coef(xv1, x1);
    float t0, t1;
    di_tau2(k0, k1, s.r, t0, t1);
    col[e0] = j0;
    cost[e0] = di_J(k0, t0);
    tau[e0] = t0;
    if (two) {
        col[e1] = j1;
        cost[e1] = di_J(k1, t1);
        tau[e1] = t1;
    }
}

// One warp evaluates the first cnt entries of its list (row v, state xv),
// written from CSR position base on: one edge per lane, two for the double
// integrator.
template <int KIND, int D, bool INCOMING>
__device__ __forceinline__ void fill_list_warp(const SpaceArgs& s, const float* __restrict__ X, const float* xv,
                                               const int* list, int cnt, int base, int* __restrict__ col,
                                               float* __restrict__ cost, float* __restrict__ tau,
                                               float* __restrict__ path) {
    const int lane = threadIdx.x & 31;
    if (KIND == GMT_COST_DI) {
        for (int t = lane; t < cnt; t += 64) {
            const bool two = t + 32 < cnt;
            fill_edge_di2<D, INCOMING>(s, X, xv, list[t], base + t, xv, list[two ? t + 32 : t], base + t + 32, two,
                                       col, cost, tau);
        }
    } else {
        for (int t = lane; t < cnt; t += 32) fill_edge<KIND, D, INCOMING>(s, X, xv, list[t], base + t, col, cost, tau, path);
    }
}

// One warp gathers row v's columns into its list (kFillList entries in shared
// memory).  A list that would overflow is evaluated by the warp on the spot;
// the entries left in it (the return value) start at CSR position *base.
template <int KIND, int D, bool INCOMING>
__device__ __forceinline__ int fill_gather(const SpaceArgs& s, const float* __restrict__ X,
                                           const uint32_t* __restrict__ M, const float* xv, int v, int* base,
                                           int* __restrict__ list, int* __restrict__ col, float* __restrict__ cost,
                                           float* __restrict__ tau, float* __restrict__ path) {
    const int lane = threadIdx.x & 31;
    const int W = (s.N + 31) / 32;
    int cnt = 0;
    // the row's words are loaded four chunks (128 words) at a time, so that one
    // latency covers rows of up to 4096 nodes
    uint32_t wb[4];
    for (int c0 = 0; c0 < W; c0 += 32) {
        const int u = (c0 >> 5) & 3;
        if (u == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int wk = c0 + 32 * k + lane;
                wb[k] = wk < W ? M[(size_t)wk * s.pitch + v] : 0u;
            }
        }
        const int w = c0 + lane;
        uint32_t bits = u == 0 ? wb[0] : u == 1 ? wb[1] : u == 2 ? wb[2] : wb[3];
        const int n = __popc(bits);
        int incl = n;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);  // at most 1024
        if (cnt + total > kFillList) {
            __syncwarp();
            fill_list_warp<KIND, D, INCOMING>(s, X, xv, list, cnt, *base, col, cost, tau, path);
            *base += cnt;
            cnt = 0;
            __syncwarp();
        }
        int pos = cnt + incl - n;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            list[pos++] = 32 * w + b;
        }
        cnt += total;
    }
    __syncwarp();
    return cnt;
}

// One warp: row v, on its own (the batched build: the warps of a block may
// belong to different queries).
template <int KIND, int D, bool INCOMING>
__device__ __forceinline__ void fill_row(const SpaceArgs& s, const float* __restrict__ X,
                                         const uint32_t* __restrict__ M, const int* __restrict__ row,
                                         int* __restrict__ col, float* __restrict__ cost, float* __restrict__ tau,
                                         float* __restrict__ path, int v, int* __restrict__ list) {
    if (v >= s.N) return;
    float xv[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xv[a] = X[(size_t)a * s.pitch + v];
    int base = row[v];
    const int cnt = fill_gather<KIND, D, INCOMING>(s, X, M, xv, v, &base, list, col, cost, tau, path);
    fill_list_warp<KIND, D, INCOMING>(s, X, xv, list, cnt, base, col, cost, tau, path);
    __syncwarp();
}

// One block: a group of kFillWarps consecutive rows of one direction.  Each
// warp gathers its row; then the block's threads share out all the group's
// listed edges, so that a row with many edges (the double integrator's slow
// states reach many more nodes than its fast ones) is spread over the block.
struct FillShared {
    int list[kFillWarps][kFillList];
    float xv[kFillWarps][GMT_MAX_DIM];
    int cnt[kFillWarps], base[kFillWarps];
    int group;
};

template <int KIND, int D, bool INCOMING>
__device__ __forceinline__ void fill_group(const SpaceArgs& s, const float* __restrict__ X, const FillDir& f,
                                           int v0, FillShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v = v0 + warp;
    int cnt = 0;
    if (v < s.N) {
        float xv[D];
#pragma unroll
        for (int a = 0; a < D; ++a) xv[a] = X[(size_t)a * s.pitch + v];
        int base = f.row[v];
        cnt = fill_gather<KIND, D, INCOMING>(s, X, f.mask, xv, v, &base, sh.list[warp], f.col, f.cost, f.tau,
                                             f.path);
        if (lane == 0) sh.base[warp] = base;
        if (lane < D) sh.xv[warp][lane] = X[(size_t)lane * s.pitch + v];
    }
    if (lane == 0) sh.cnt[warp] = cnt;
    __syncthreads();
    // the group's entries in warp order: entry k is list[w][k - pre[w]]
    int pre[kFillWarps + 1];
    pre[0] = 0;
#pragma unroll
    for (int w = 0; w < kFillWarps; ++w) pre[w + 1] = pre[w] + sh.cnt[w];
    const int T = pre[kFillWarps];
    auto locate = [&](int k, int& w, int& t) {  // selects only: pre[] stays in registers
        int pw = 0;
        w = 0;
#pragma unroll
        for (int u = 1; u < kFillWarps; ++u)
            if (k >= pre[u]) { w = u; pw = pre[u]; }
        t = k - pw;
    };
    constexpr int kT = kFillWarps * 32;
    if (KIND == GMT_COST_DI) {
        for (int k0 = threadIdx.x; k0 < T; k0 += 2 * kT) {
            const int k1 = k0 + kT;
            const bool two = k1 < T;
            int w0, t0, w1, t1;
            locate(k0, w0, t0);
            locate(two ? k1 : k0, w1, t1);
            float xv0[D], xv1[D];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                xv0[a] = sh.xv[w0][a];
                xv1[a] = sh.xv[w1][a];
            }
            fill_edge_di2<D, INCOMING>(s, X, xv0, sh.list[w0][t0], sh.base[w0] + t0, xv1, sh.list[w1][t1],
                                       sh.base[w1] + t1, two, f.col, f.cost, f.tau);
        }
    } else {
        for (int k = threadIdx.x; k < T; k += kT) {
            int w, t;
            locate(k, w, t);
            float xv[D];
#pragma unroll
            for (int a = 0; a < D; ++a) xv[a] = sh.xv[w][a];
            fill_edge<KIND, D, INCOMING>(s, X, xv, sh.list[w][t], sh.base[w] + t, f.col, f.cost, f.tau, f.path);
        }
    }
    __syncthreads();  // the lists are refilled by the next group
}

}  // namespace gmtk
