// Cell-list neighbour build for one graph (kernels in cells_body.cuh).
#include <cmath>

#include "cells_body.cuh"

namespace gmtk {

template <int D>
__global__ void __launch_bounds__(256) cells_count_kernel(SpaceArgs s, const float* __restrict__ X, CellGrid cg,
                                                          int* __restrict__ cell_of, int* __restrict__ cnt) {
    cell_count_node<D>(s, X, cg, cell_of, cnt, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256) cells_scatter_kernel(int N, const int* __restrict__ cell_of,
                                                            const int* __restrict__ start, int* __restrict__ cnt,
                                                            int* __restrict__ sorted) {
    cell_scatter_node(N, cell_of, start, cnt, sorted, blockIdx.x * blockDim.x + threadIdx.x);
}

template <int D, bool FILL>
__global__ void __launch_bounds__(kCellWarps * 32) cells_tile_kernel(SpaceArgs s, const float* __restrict__ X,
                                                                     CellGrid cg, const int* __restrict__ start,
                                                                     const int* __restrict__ sorted,
                                                                     int* __restrict__ out_count,
                                                                     int* __restrict__ max_deg,
                                                                     const int* __restrict__ row,
                                                                     int* __restrict__ col, float* __restrict__ cost,
                                                                     int* __restrict__ overflow, int words) {
    extern __shared__ int cell_buf[];
    cell_tile<D, FILL>(s, X, cg, start, sorted, out_count, max_deg, row, col, cost, overflow, cell_buf, words,
                       blockIdx.x);
}

// ---- box grid (checks against many boxes)
// The cell range [c0, c1] of box b on the grid's axes (empty when lo > hi).
__device__ __forceinline__ void box_grid_range(const BoxGridArgs& g, const float* lo, const float* hi, int* c0,
                                               int* c1) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        c0[a] = box_grid_cell(g, lo[a], a);
        c1[a] = box_grid_cell(g, hi[a], a);
    }
}

// One thread per box: counts it in each cell it overlaps, or lists it as big.
__global__ void __launch_bounds__(256) box_grid_count_kernel(BoxArgs boxes, int dp, BoxGridArgs grid,
                                                             int* __restrict__ cnt, int* __restrict__ big,
                                                             int* __restrict__ nbig) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= boxes.count) return;
    int c0[2], c1[2];
    box_grid_range(grid, boxes.lo + (size_t)b * dp, boxes.hi + (size_t)b * dp, c0, c1);
    if (c0[0] > c1[0] || c0[1] > c1[1]) return;  // lo > hi: the box holds no point
    if ((c1[0] - c0[0] + 1) * (c1[1] - c0[1] + 1) > kBoxGridMaxCells) {
        big[atomicAdd(nbig, 1)] = b;
        return;
    }
    for (int cy = c0[1]; cy <= c1[1]; ++cy)
        for (int cx = c0[0]; cx <= c1[0]; ++cx) atomicAdd(&cnt[cy * grid.g + cx], 1);
}

// One thread per box: writes it into each of its cells' lists (cnt counts
// back down to 0).
__global__ void __launch_bounds__(256) box_grid_scatter_kernel(BoxArgs boxes, int dp, BoxGridArgs grid,
                                                               const int* __restrict__ start, int* __restrict__ cnt,
                                                               int* __restrict__ list) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= boxes.count) return;
    int c0[2], c1[2];
    box_grid_range(grid, boxes.lo + (size_t)b * dp, boxes.hi + (size_t)b * dp, c0, c1);
    if (c0[0] > c1[0] || c0[1] > c1[1]) return;
    if ((c1[0] - c0[0] + 1) * (c1[1] - c0[1] + 1) > kBoxGridMaxCells) return;
    for (int cy = c0[1]; cy <= c1[1]; ++cy)
        for (int cx = c0[0]; cx <= c1[0]; ++cx) {
            const int c = cy * grid.g + cx;
            list[start[c] + atomicSub(&cnt[c], 1) - 1] = b;
        }
}

cudaError_t launch_box_grid(int dp, BoxArgs boxes, const BoxGridArgs& grid, int* cnt, int* start, int* list,
                            int* big, int* nbig, cudaStream_t st) {
    if (dp < 2 || boxes.count < 1) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((boxes.count + 255) / 256);
    box_grid_count_kernel<<<blocks, 256, 0, st>>>(boxes, dp, grid, cnt, big, nbig);
    cudaError_t e = launch_scan(cnt, start, grid.g * grid.g, st);
    if (e != cudaSuccess) return e;
    box_grid_scatter_kernel<<<blocks, 256, 0, st>>>(boxes, dp, grid, start, cnt, list);
    return cudaGetLastError();
}

bool make_cell_grid(int kind, int d, const float* lo, const float* hi, float r, int N, bool batched, CellGrid* cg,
                    bool* pays) {
    if (kind != GMT_COST_EUCLID || (d != 2 && d != 3) || !(r > 0.0f)) return false;
    // cell side: at least 1.01 r, and coarse enough for at most 2^16 cells
    double h = (double)r * 1.01;
    for (;;) {
        double cells = 1.0;
        for (int a = 0; a < d; ++a) cells *= std::floor(((double)hi[a] - (double)lo[a]) / h) + 1.0;
        if (cells <= 65536.0) break;
        h *= 1.25;
    }
    double frac = 1.0;
    long long ncells = 1;
    for (int a = 0; a < 3; ++a) {
        cg->g[a] = 1;
        cg->lo[a] = 0.0f;
        if (a >= d) continue;
        const double L = (double)hi[a] - (double)lo[a];
        cg->g[a] = (int)std::floor(L / h) + 1;
        cg->lo[a] = lo[a];
        frac *= std::min(1.0, 3.0 * h / L);
        ncells *= cg->g[a];
    }
    // keep h >= 1.01 r for the rounded reciprocal too
    cg->inv_h = (float)(1.0 / h);
    while ((double)r * 1.01 * (double)cg->inv_h > 1.0) cg->inv_h = std::nextafter(cg->inv_h, 0.0f);
    cg->ncells = (int)ncells;
    cg->list_only = 0;
    // measured on one GB300 (Theorem 1 radii, cell tiles against the packed
    // all-pairs test and the tiled fill): on one graph in 2D the cell list
    // loses at 8192 nodes (0.055 against 0.040 ms) and wins at 16384 (0.069
    // against 0.087); in a batch (where the cell stages' short launches
    // overlap other queries' work) it already pays from 4096; in 3D, with 27
    // cells of candidates to sort per tile, it loses at 16384 (0.216 against
    // 0.113 ms) and wins at 32768 (0.280 against 0.388)
    *pays = frac <= 0.25 && N >= (d == 2 ? (batched ? 4096 : 12000) : 32768);
    return true;
}

namespace {
template <int D>
cudaError_t rows_t(const SpaceArgs& s, const float* X, const CellGrid& cg, const int* start, const int* sorted,
                   bool fill, int* out_count, int* max_deg, const int* row, int* col, float* cost, int* overflow,
                   cudaStream_t st) {
    const int words = fill ? cell_fill_words(cg, s.N) : 0;
    const size_t smem = cell_tile_smem(D, words);
    if (fill)
        cells_tile_kernel<D, true><<<cg.ncells, kCellWarps * 32, smem, st>>>(s, X, cg, start, sorted, out_count,
                                                                             max_deg, row, col, cost, overflow, words);
    else
        cells_tile_kernel<D, false><<<cg.ncells, kCellWarps * 32, smem, st>>>(s, X, cg, start, sorted, out_count,
                                                                              max_deg, row, col, cost, overflow, 0);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_cells_count(const SpaceArgs& s, const float* X, const CellGrid& cg, int* cell_of, int* cell_cnt,
                               cudaStream_t st) {
    const int blocks = (s.N + 255) / 256;
    if (s.d == 2) cells_count_kernel<2><<<blocks, 256, 0, st>>>(s, X, cg, cell_of, cell_cnt);
    else if (s.d == 3) cells_count_kernel<3><<<blocks, 256, 0, st>>>(s, X, cg, cell_of, cell_cnt);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_cells_scatter(int N, const int* cell_of, const int* cell_start, int* cell_cnt, int* sorted,
                                 cudaStream_t st) {
    cells_scatter_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, cell_of, cell_start, cell_cnt, sorted);
    return cudaGetLastError();
}

cudaError_t launch_cells_rows(const SpaceArgs& s, const float* X, const CellGrid& cg, const int* cell_of,
                              const int* cell_start, const int* sorted, bool fill, int* out_count, int* max_deg,
                              const int* row, int* col, float* cost, int* overflow, cudaStream_t st) {
    (void)cell_of;
    if (s.d == 2) return rows_t<2>(s, X, cg, cell_start, sorted, fill, out_count, max_deg, row, col, cost, overflow, st);
    if (s.d == 3) return rows_t<3>(s, X, cg, cell_start, sorted, fill, out_count, max_deg, row, col, cost, overflow, st);
    return cudaErrorInvalidValue;
}

}  // namespace gmtk
