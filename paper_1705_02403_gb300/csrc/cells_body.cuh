// Cell-list neighbour search for geometric graphs in 2 and 3 dimensions: a
// faster way to the same neighbour sets (Section III-A's r-disk neighbours,
// precomputed in Section V-A), not a change of the method.  Nodes are
// counting-sorted by grid cell; a row's candidates are the nodes of the 3^d
// cells around its own, which lie in 3^(d-1) runs of consecutive cells along
// axis 0.  Every candidate takes the same FP32 edge predicate as the all-pairs
// build, and each row's columns come out in ascending order, so the CSR is the
// same bits.
//
// One CTA per cell (a cell tile): the cell's candidates (the same for every
// row of the cell) are loaded into shared memory once, with their
// coordinates, and for the fill sorted by node index (bitonic); then each warp
// takes rows of the cell and tests 32 candidates per step, so a row's passing
// candidates come out in ascending order from a ballot and are written
// straight into the CSR.  A cell with more than kTileCand candidates takes the
// row-by-row path instead (one warp per row, candidates gathered from global
// memory, columns ordered through a bitmap of the row or a sorted list).
#pragma once

#include "graph_body.cuh"

namespace gmtk {

constexpr int kCellWarps = 8;    // warps per cell tile
constexpr int kTileCand = 2048;  // candidates a cell tile holds in shared memory

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

// Words of the row-by-row fill's per-warp buffer for a graph of N nodes.
__host__ __device__ inline int cell_fill_words(const CellGrid& cg, int N) {
    const int W = (N + 31) / 32;
    return !cg.list_only && W <= kCellList ? W : kCellList;
}

// Dynamic shared memory of a cell tile: the candidate tile or, for a cell
// with too many candidates, the row-by-row buffers of its warps.
__host__ __device__ inline size_t cell_tile_smem(int D, int words) {
    const size_t tile = (size_t)kTileCand * (1 + D) * sizeof(int);
    const size_t rows = (size_t)kCellWarps * words * sizeof(int);
    return tile > rows ? tile : rows;
}

// The candidate runs of cell `cell`: up to 3^(d-1) runs of consecutive cells
// along axis 0 ([rs, re) in the cell-sorted node order).  Returns their total.
template <int D>
__device__ __forceinline__ int cell_runs(const CellGrid& cg, const int* __restrict__ start, int cell, int* rs,
                                         int* re) {
    constexpr int NR = D == 3 ? 9 : 3;
    int c[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        c[a] = cell % cg.g[a];
        cell /= cg.g[a];
    }
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
    return T;
}

// Candidate t of the runs (t < their total).
template <int D>
__device__ __forceinline__ int run_candidate(const int* __restrict__ sorted, const int* rs, const int* re, int t) {
    constexpr int NR = D == 3 ? 9 : 3;
    int j = -1, off = t;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int len = re[k] - rs[k];
        if (j < 0 && off >= 0 && off < len) j = sorted[rs[k] + off];
        off -= len;
    }
    return j;
}

// Row-by-row path, one warp: row v with candidates in the given runs.  Count
// pass (FILL = false) or fill pass, whose warp buffer `list` holds
// cell_fill_words(cg, N) words.
template <int D, bool FILL>
__device__ __forceinline__ void cell_row(const SpaceArgs& s, const float* __restrict__ X, const CellGrid& cg,
                                         const int* __restrict__ sorted, const int* rs, const int* re, int T,
                                         int* __restrict__ out_count, int* __restrict__ max_deg,
                                         const int* __restrict__ row, int* __restrict__ col, float* __restrict__ cost,
                                         int* __restrict__ overflow, int* list, int v) {
    const int lane = threadIdx.x & 31;
    float xv[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xv[a] = X[(size_t)a * s.pitch + v];
    // Fill: with N <= 32 kCellList the warp's buffer holds a bitmap of the
    // row's columns, which yields them in ascending order; larger graphs keep
    // a list of columns and sort it (bitonic).
    const int W = (s.N + 31) / 32;
    const bool bitmap = FILL && W <= kCellList && !cg.list_only;
    if (bitmap) {
        for (int q = lane; q < W; q += 32) list[q] = 0;
        __syncwarp();
    }
    int n = 0;
    for (int t0 = 0; t0 < T; t0 += 32) {
        const int t = t0 + lane;
        const int j = t < T ? run_candidate<D>(sorted, rs, re, t) : -1;
        bool pass = false;
        if (j >= 0 && j != v) {
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
            const int wd = c0 + lane;
            unsigned bits = wd < W ? (unsigned)list[wd] : 0u;
            const int cnt = __popc(bits);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int pos = b + done + incl - cnt;
            while (bits) {
                const int j = 32 * wd + __ffs(bits) - 1;
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

// One CTA of kCellWarps warps: every row of cell `cell`.  smem:
// cell_tile_smem(D, words) bytes; words = cell_fill_words(cg, N) (fill).
template <int D, bool FILL>
__device__ __forceinline__ void cell_tile(const SpaceArgs& s, const float* __restrict__ X, const CellGrid& cg,
                                          const int* __restrict__ start, const int* __restrict__ sorted,
                                          int* __restrict__ out_count, int* __restrict__ max_deg,
                                          const int* __restrict__ row, int* __restrict__ col,
                                          float* __restrict__ cost, int* __restrict__ overflow, int* smem, int words,
                                          int cell) {
    constexpr int NR = D == 3 ? 9 : 3;
    const int r0 = start[cell], R = start[cell + 1] - r0;
    if (R <= 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int rs[NR], re[NR];
    const int T = cell_runs<D>(cg, start, cell, rs, re);
    if (T > kTileCand) {
        for (int r = warp; r < R; r += kCellWarps)
            cell_row<D, FILL>(s, X, cg, sorted, rs, re, T, out_count, max_deg, row, col, cost, overflow,
                              smem + warp * words, sorted[r0 + r]);
        return;
    }
    int* cand = smem;
    float* xs = (float*)(smem + kTileCand);  // xs[a * kTileCand + t]
    int L = T;
    if (FILL) {  // sort the candidates by node index (bitonic, padded with INT_MAX)
        L = 1;
        while (L < T) L <<= 1;
    }
    for (int t = threadIdx.x; t < L; t += blockDim.x)
        cand[t] = t < T ? run_candidate<D>(sorted, rs, re, t) : INT_MAX;
    __syncthreads();
    if (FILL) {
        for (int k = 2; k <= L; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = threadIdx.x; i < L; i += blockDim.x) {
                    const int ix = i ^ jj;
                    if (ix > i) {
                        const int a = cand[i], b2 = cand[ix];
                        if ((a > b2) == ((i & k) == 0)) {
                            cand[i] = b2;
                            cand[ix] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const int j = cand[t];
#pragma unroll
        for (int a = 0; a < D; ++a) xs[a * kTileCand + t] = X[(size_t)a * s.pitch + j];
    }
    __syncthreads();
    int longest = 0;
    for (int r = warp; r < R; r += kCellWarps) {
        const int v = sorted[r0 + r];
        float xv[D];
#pragma unroll
        for (int a = 0; a < D; ++a) xv[a] = X[(size_t)a * s.pitch + v];
        const int b = FILL ? row[v] : 0, e = FILL ? row[v + 1] : 0;
        int n = 0;
        for (int t0 = 0; t0 < T; t0 += 32) {
            const int t = t0 + lane;
            bool pass = false;
            int j = -1;
            float xj[D];
            if (t < T) {
                j = cand[t];
#pragma unroll
                for (int a = 0; a < D; ++a) xj[a] = xs[a * kTileCand + t];
                pass = j != v && connects<GMT_COST_EUCLID, D>(s, xv, xj);
            }
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            if (FILL && pass) {
                const int pos = b + n + __popc(m & ((1u << lane) - 1u));
                if (pos < e) {
                    col[pos] = j;
                    cost[pos] = edge_cost<GMT_COST_EUCLID, D>(s, xv, xj);
                }
            }
            n += __popc(m);
        }
        if (!FILL && lane == 0) out_count[v] = n;
        longest = max(longest, n);
    }
    if (!FILL && lane == 0 && longest > 0) atomicMax(max_deg, longest);
}

}  // namespace gmtk
