// SampleFree and r-disk neighbour graph construction (Section III-B; the
// precomputation of Section V-A), as CUDA kernels for sm_103a.
//
//   sample_kernel     one thread per node: Philox4x32-10 rejection sampling
//   pair_mask_kernel  all ordered pairs (i, j): bit j of row i is set iff
//                     c(i, j) < r; rows staged through shared memory; the bit
//                     matrix is word-major (word w of every row contiguous) so
//                     that each warp writes 32 consecutive rows' words
//   transpose_kernel  32x32 bit-block transpose with warp ballots (in-edges)
//   scan_kernel       exclusive prefix sum of the per-row counts -> row_ptr
//   fill_kernel       one warp per row: ballot-free prefix over the row's
//                     words, costs of the set bits, ascending column order
#include <cstdio>

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
__global__ void __launch_bounds__(128) sample_kernel(SpaceArgs s, BoxArgs boxes, float* __restrict__ X,
                                                     uint8_t* __restrict__ is_goal, int* __restrict__ flags) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.N) return;
    float x[D];
    if (k == 0) {
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            x[a] = s.x0[a];
            ok = ok && s.lo[a] <= x[a] && x[a] <= s.hi[a];
        }
        if (!ok || in_any_box<DP>(x, boxes.lo, boxes.hi, boxes.count)) atomicOr(flags, kSampleBadInit);
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
            if (in_any_box<DP>(x, boxes.lo, boxes.hi, boxes.count)) continue;
            ok = true;
        }
        if (!ok) atomicOr(flags, kSampleExhausted);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) X[(size_t)a * s.pitch + k] = x[a];
    is_goal[k] = in_goal_ball(x, s.gd, s.gc, s.grho) ? 1 : 0;
}

// ------------------------------------------------------------- pair filter
constexpr int kMaskRows = 256;     // rows (threads) per block
constexpr int kMaskWords = 8;      // 32-column words per block (256 columns staged in shared memory)

template <int KIND, int D>
__device__ __forceinline__ bool connects(const SpaceArgs& s, const float* from, const float* to) {
    if (KIND == GMT_COST_EUCLID) return sq_dist<D>(from, to) < s.r2_threshold;
    if (!di_may_connect(from, to, s.r)) return false;
    return di_cost(from, to, s.r) < s.r;
}

template <int KIND, int D>
__device__ __forceinline__ float edge_cost(const SpaceArgs& s, const float* from, const float* to) {
    if (KIND == GMT_COST_EUCLID) return __fsqrt_rn(sq_dist<D>(from, to));
    return di_cost(from, to, s.r);
}

template <int KIND, int D>
__global__ void __launch_bounds__(kMaskRows) pair_mask_kernel(SpaceArgs s, const float* __restrict__ X,
                                                              uint32_t* __restrict__ mask,
                                                              int* __restrict__ out_count) {
    __shared__ float tile[D][kMaskWords * 32];
    const int i = blockIdx.x * kMaskRows + threadIdx.x;
    const int w0 = blockIdx.y * kMaskWords;
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

// maskT[u][j] bit l = mask[j/32][32u + l] bit (j%32): the in-neighbour rows.
__global__ void __launch_bounds__(256) transpose_kernel(int N, int pitch, const uint32_t* __restrict__ mask,
                                                        uint32_t* __restrict__ maskT, int* __restrict__ in_count) {
    const int W = (N + 31) / 32;
    const long long task = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
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

// Exclusive prefix sum: row[v] = sum_{u < v} count[u], row[N] = total.
__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ count, int* __restrict__ row, int N) {
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
}

// One warp per row v: words of the row's bits are read 32 at a time, the
// lanes' edge counts are prefix-summed, and each lane writes the edges of its
// word (ascending column order overall).
template <int KIND, int D, bool INCOMING>
__global__ void __launch_bounds__(256) fill_kernel(SpaceArgs s, const float* __restrict__ X,
                                                   const uint32_t* __restrict__ M, const int* __restrict__ row,
                                                   int* __restrict__ col, float* __restrict__ cost) {
    const int v = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32);
    const int lane = threadIdx.x & 31;
    if (v >= s.N) return;
    float xv[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xv[a] = X[(size_t)a * s.pitch + v];
    const int W = (s.N + 31) / 32;
    int base = row[v];
    for (int c0 = 0; c0 < W; c0 += 32) {
        const int w = c0 + lane;
        uint32_t bits = w < W ? M[(size_t)w * s.pitch + v] : 0u;
        const int n = __popc(bits);
        int incl = n;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        int pos = base + incl - n;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int j = 32 * w + b;
            float xj[D];
#pragma unroll
            for (int a = 0; a < D; ++a) xj[a] = X[(size_t)a * s.pitch + j];
            col[pos] = j;
            cost[pos] = INCOMING ? edge_cost<KIND, D>(s, xj, xv) : edge_cost<KIND, D>(s, xv, xj);
            ++pos;
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// ------------------------------------------------------------------ launchers
namespace {
template <int D, int DP>
cudaError_t sample_t(const SpaceArgs& s, BoxArgs b, float* X, uint8_t* g, int* f, cudaStream_t st) {
    sample_kernel<D, DP><<<(s.N + 127) / 128, 128, 0, st>>>(s, b, X, g, f);
    return cudaGetLastError();
}
template <int KIND, int D>
cudaError_t mask_t(const SpaceArgs& s, const float* X, uint32_t* mask, int* cnt, cudaStream_t st) {
    const int W = (s.N + 31) / 32;
    dim3 grid((s.N + kMaskRows - 1) / kMaskRows, (W + kMaskWords - 1) / kMaskWords);
    pair_mask_kernel<KIND, D><<<grid, kMaskRows, 0, st>>>(s, X, mask, cnt);
    return cudaGetLastError();
}
template <int KIND, int D>
cudaError_t fill_t(const SpaceArgs& s, const float* X, const uint32_t* M, const int* row, int* col, float* cost,
                   bool incoming, cudaStream_t st) {
    const long long threads = (long long)s.N * 32;
    const int blocks = (int)((threads + 255) / 256);
    if (incoming) fill_kernel<KIND, D, true><<<blocks, 256, 0, st>>>(s, X, M, row, col, cost);
    else fill_kernel<KIND, D, false><<<blocks, 256, 0, st>>>(s, X, M, row, col, cost);
    return cudaGetLastError();
}
}  // namespace

#define GMT_EUCLID_DIMS(F, ...)                                      \
    switch (s.d) {                                                   \
        case 2: return F<GMT_COST_EUCLID, 2>(__VA_ARGS__);           \
        case 3: return F<GMT_COST_EUCLID, 3>(__VA_ARGS__);           \
        case 4: return F<GMT_COST_EUCLID, 4>(__VA_ARGS__);           \
        case 5: return F<GMT_COST_EUCLID, 5>(__VA_ARGS__);           \
        case 6: return F<GMT_COST_EUCLID, 6>(__VA_ARGS__);           \
        case 7: return F<GMT_COST_EUCLID, 7>(__VA_ARGS__);           \
        case 8: return F<GMT_COST_EUCLID, 8>(__VA_ARGS__);           \
        case 9: return F<GMT_COST_EUCLID, 9>(__VA_ARGS__);           \
        case 10: return F<GMT_COST_EUCLID, 10>(__VA_ARGS__);         \
        default: return cudaErrorInvalidValue;                       \
    }

cudaError_t launch_sample(const SpaceArgs& s, BoxArgs b, float* X, uint8_t* g, int* f, cudaStream_t st) {
    if (s.kind == GMT_COST_DI) return sample_t<6, 3>(s, b, X, g, f, st);
    switch (s.d) {
        case 2: return sample_t<2, 2>(s, b, X, g, f, st);
        case 3: return sample_t<3, 3>(s, b, X, g, f, st);
        case 4: return sample_t<4, 4>(s, b, X, g, f, st);
        case 5: return sample_t<5, 5>(s, b, X, g, f, st);
        case 6: return sample_t<6, 6>(s, b, X, g, f, st);
        case 7: return sample_t<7, 7>(s, b, X, g, f, st);
        case 8: return sample_t<8, 8>(s, b, X, g, f, st);
        case 9: return sample_t<9, 9>(s, b, X, g, f, st);
        case 10: return sample_t<10, 10>(s, b, X, g, f, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pair_mask(const SpaceArgs& s, const float* X, uint32_t* mask, int* cnt, cudaStream_t st) {
    if (s.kind == GMT_COST_DI) return mask_t<GMT_COST_DI, 6>(s, X, mask, cnt, st);
    GMT_EUCLID_DIMS(mask_t, s, X, mask, cnt, st)
}

cudaError_t launch_transpose(const SpaceArgs& s, const uint32_t* mask, uint32_t* maskT, int* in_count,
                             cudaStream_t st) {
    const long long W = (s.N + 31) / 32;
    const long long threads = W * W * 32;
    transpose_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(s.N, s.pitch, mask, maskT, in_count);
    return cudaGetLastError();
}

cudaError_t launch_scan(const int* count, int* row, int N, cudaStream_t st) {
    scan_kernel<<<1, 1024, 0, st>>>(count, row, N);
    return cudaGetLastError();
}

cudaError_t launch_fill(const SpaceArgs& s, const float* X, const uint32_t* M, const int* row, int* col,
                        float* cost, bool incoming, cudaStream_t st) {
    if (s.kind == GMT_COST_DI) return fill_t<GMT_COST_DI, 6>(s, X, M, row, col, cost, incoming, st);
    GMT_EUCLID_DIMS(fill_t, s, X, M, row, col, cost, incoming, st)
}

}  // namespace gmtk
