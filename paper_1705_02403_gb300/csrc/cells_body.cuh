// Cell-list neighbour search for geometric graphs in 2 and 3 dimensions: a
// faster way to the same neighbour sets (Section III-A's r-disk neighbours,
// precomputed in Section V-A), not a change of the method.  Nodes are
// counting-sorted by grid cell; a row's candidates are the nodes of the 3^d
// cells around its own, which lie in 3^(d-1) runs of consecutive cells along
// axis 0.  Every candidate takes the same FP32 edge predicate as the all-pairs
// build, and each row's columns come out in ascending order (a bitmap of the
// row in shared memory, or a bitonic sort for graphs beyond 32768 nodes), so
// the CSR is the same bits.
#pragma once

#include "graph_body.cuh"

namespace gmtk {

constexpr int kCellWarps = 8;  // rows (one per warp) per block

template <int D>
__device__ __forceinline__ int cell_index(const CellGrid& cg, const float* x) {
    int idx = 0;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
        int k = (int)floorf((x[a] - cg.lo[a]) * cg.inv_h);
        k = min(max(k, 0), cg.g[a] - 1);
        idx = idx * cg.g[a] + k;
    }
    return idx;
}

template <int D>
__device__ __forceinline__ void cell_count_node(const SpaceArgs& s, const float* __restrict__ X, const CellGrid& cg,
                                                int* __restrict__ cell_of, int* __restrict__ cnt, int v) {
    if (v >= s.N) return;
    float x[D];
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = X[(size_t)a * s.pitch + v];
    const int c = cell_index<D>(cg, x);
    cell_of[v] = c;
    atomicAdd(&cnt[c], 1);
}

__device__ __forceinline__ void cell_scatter_node(int N, const int* __restrict__ cell_of,
                                                  const int* __restrict__ start, int* __restrict__ cnt,
                                                  int* __restrict__ sorted, int v) {
    if (v >= N) return;
    const int c = cell_of[v];
    sorted[start[c] + atomicSub(&cnt[c], 1) - 1] = v;
}

// Words of the fill's per-warp shared-memory buffer for a graph of N nodes.
__host__ __device__ inline int cell_fill_words(const CellGrid& cg, int N) {
    const int W = (N + 31) / 32;
    return !cg.list_only && W <= kCellList ? W : kCellList;
}

// One warp: row v.  Count pass (FILL = false) or fill pass, whose warp buffer
// `list` holds cell_fill_words(cg, N) words (only what the row needs, so that
// the rest of the SM's L1 keeps caching the samples).
template <int D, bool FILL>
__device__ __forceinline__ void cell_row(const SpaceArgs& s, const float* __restrict__ X, const CellGrid& cg,
                                         const int* __restrict__ cell_of, const int* __restrict__ start,
                                         const int* __restrict__ sorted, int* __restrict__ out_count,
                                         int* __restrict__ max_deg, const int* __restrict__ row,
                                         int* __restrict__ col, float* __restrict__ cost, int* __restrict__ overflow,
                                         int* list, int v) {
    constexpr int NR = D == 3 ? 9 : 3;  // runs of up to 3 cells along axis 0
    const int lane = threadIdx.x & 31;
    if (v >= s.N) return;
    float xv[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xv[a] = X[(size_t)a * s.pitch + v];
    int c[3] = {0, 0, 0};
    {
        int idx = cell_of[v];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            c[a] = idx % cg.g[a];
            idx /= cg.g[a];
        }
    }
    int rs[NR], re[NR];
    int T = 0;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int y = c[1] + (k % 3) - 1, z = D == 3 ? c[2] + (k / 3) - 1 : 0;
        const bool ok = y >= 0 && y < cg.g[1] && z >= 0 && z < cg.g[2];
        const int base = (z * cg.g[1] + y) * cg.g[0];
        const int x0 = max(c[0] - 1, 0), x1 = min(c[0] + 1, cg.g[0] - 1);
        rs[k] = ok ? start[base + x0] : 0;
        re[k] = ok ? start[base + x1 + 1] : 0;
        T += re[k] - rs[k];
    }
    // Fill: with N <= 32 kCellList the warp's buffer holds a bitmap of the
    // row's columns, which yields them in ascending order; larger graphs keep
    // a list of columns and sort it (bitonic).
    const int W = (s.N + 31) / 32;
    const bool bitmap = FILL && W <= kCellList && !cg.list_only;
    if (bitmap) {
        for (int w = lane; w < W; w += 32) list[w] = 0;
        __syncwarp();
    }
    int n = 0;
    for (int t0 = 0; t0 < T; t0 += 32) {
        const int t = t0 + lane;
        int j = -1, off = t;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const int len = re[k] - rs[k];
            if (j < 0 && off >= 0 && off < len) j = sorted[rs[k] + off];
            off -= len;
        }
        bool pass = false;
        if (t < T && j >= 0 && j != v) {
            float xj[D];
#pragma unroll
            for (int a = 0; a < D; ++a) xj[a] = X[(size_t)a * s.pitch + j];
            pass = connects<GMT_COST_EUCLID, D>(s, xv, xj);
        }
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        if (bitmap) {
            if (pass) atomicOr((unsigned*)&list[j >> 5], 1u << (j & 31));
        } else if (FILL) {
            const int pos = n + __popc(m & ((1u << lane) - 1u));
            if (pass && pos < kCellList) list[pos] = j;
        }
        n += __popc(m);
    }
    if (!FILL) {
        if (lane == 0) {
            out_count[v] = n;
            atomicMax(max_deg, n);
        }
        return;
    }
    const int b = row[v];
    if (bitmap) {
        __syncwarp();
        int done = 0;
        for (int c0 = 0; c0 < W; c0 += 32) {
            const int w = c0 + lane;
            unsigned bits = w < W ? (unsigned)list[w] : 0u;
            const int cnt = __popc(bits);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int pos = b + done + incl - cnt;
            while (bits) {
                const int j = 32 * w + __ffs(bits) - 1;
                bits &= bits - 1;
                float xj[D];
#pragma unroll
                for (int a = 0; a < D; ++a) xj[a] = X[(size_t)a * s.pitch + j];
                col[pos] = j;
                cost[pos] = edge_cost<GMT_COST_EUCLID, D>(s, xv, xj);
                ++pos;
            }
            done += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
        return;
    }
    if (n > kCellList) {
        if (lane == 0) atomicExch(overflow, 1);
        return;
    }
    // bitonic sort of the row's columns (padded to a power of two with INT_MAX)
    int L = 1;
    while (L < n) L <<= 1;
    for (int t = n + lane; t < L; t += 32) list[t] = INT_MAX;
    __syncwarp();
    for (int k = 2; k <= L; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = lane; i < L; i += 32) {
                const int ix = i ^ jj;
                if (ix > i) {
                    const int a = list[i], b2 = list[ix];
                    if ((a > b2) == ((i & k) == 0)) {
                        list[i] = b2;
                        list[ix] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
    for (int t = lane; t < n; t += 32) {
        const int j = list[t];
        float xj[D];
#pragma unroll
        for (int a = 0; a < D; ++a) xj[a] = X[(size_t)a * s.pitch + j];
        col[b + t] = j;
        cost[b + t] = edge_cost<GMT_COST_EUCLID, D>(s, xv, xj);
    }
    __syncwarp();
}

}  // namespace gmtk
