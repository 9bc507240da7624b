// Cell-list neighbour search for geometric graphs in 2 and 3 dimensions (an
// acceleration of the all-pairs neighbour test of Section III-A; Section VI
// names spatial data structures as the way to large sample counts).  Nodes are
// counting-sorted by grid cell; a row's candidates are the nodes of the 3^d
// cells around its own, which lie in 3^(d-1) runs of consecutive cells along
// axis 0.  Every candidate takes the same FP32 edge predicate as the all-pairs
// build, and each row's columns are sorted, so the CSR is the same bits.
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

// One warp: row v.  Count pass (FILL = false) or fill pass.
template <int D, bool FILL>
__device__ __forceinline__ void cell_row(const SpaceArgs& s, const float* __restrict__ X, const CellGrid& cg,
                                         const int* __restrict__ cell_of, const int* __restrict__ start,
                                         const int* __restrict__ sorted, int* __restrict__ out_count,
                                         int* __restrict__ max_deg, const int* __restrict__ row,
                                         int* __restrict__ col, float* __restrict__ cost, int* __restrict__ overflow,
                                         int v) {
    __shared__ int list[kCellWarps][kCellList];
    constexpr int NR = D == 3 ? 9 : 3;  // runs of up to 3 cells along axis 0
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
        if (FILL) {
            const int pos = n + __popc(m & ((1u << lane) - 1u));
            if (pass && pos < kCellList) list[warp][pos] = j;
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
    if (n > kCellList) {
        if (lane == 0) atomicExch(overflow, 1);
        return;
    }
    __syncwarp();
    const int b = row[v];
    for (int t = lane; t < n; t += 32) {
        const int j = list[warp][t];
        int rank = 0;
        for (int u = 0; u < n; ++u) rank += list[warp][u] < j;
        float xj[D];
#pragma unroll
        for (int a = 0; a < D; ++a) xj[a] = X[(size_t)a * s.pitch + j];
        col[b + rank] = j;
        cost[b + rank] = edge_cost<GMT_COST_EUCLID, D>(s, xv, xj);
    }
    __syncwarp();
}

}  // namespace gmtk
