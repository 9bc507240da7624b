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
//   pair_mask_di_kernel  the same for the double integrator, with a
//                     conservative lower bound and per-warp compaction of the
//                     pairs that need the exact root procedure
//   fill_kernel       one warp per row: prefix over the row's words, column
//                     list in shared memory, one edge cost per lane
#include <cstdio>

#include "graph_body.cuh"

namespace gmtk {

// ------------------------------------------------------------------ kernels
template <int D, int DP>
__global__ void __launch_bounds__(128) sample_kernel(SpaceArgs s, BoxArgs boxes, float* __restrict__ X,
                                                     uint8_t* __restrict__ is_goal, int* __restrict__ flags) {
    sample_node<D, DP>(s, boxes, X, is_goal, flags, blockIdx.x * blockDim.x + threadIdx.x);
}

template <int D, int DP>
__global__ void __launch_bounds__(128) append_kernel(SpaceArgs s, BoxArgs boxes, const float* __restrict__ src,
                                                     int src_pitch, int first, int count, float* __restrict__ X,
                                                     uint8_t* __restrict__ is_goal, int* __restrict__ flags) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) append_node<D, DP>(s, boxes, src, src_pitch, first, X, is_goal, flags, k);
}

template <int KIND, int D>
__global__ void __launch_bounds__(kMaskRows) pair_mask_kernel(SpaceArgs s, const float* __restrict__ X,
                                                              uint32_t* __restrict__ mask,
                                                              int* __restrict__ out_count) {
    mask_tile<KIND, D>(s, X, mask, out_count, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(kDIRows, 8) pair_mask_di_kernel(SpaceArgs s, const float* __restrict__ X,
                                                              uint32_t* __restrict__ mask,
                                                              int* __restrict__ out_count) {
    mask_di_tile(s, X, mask, out_count, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(256) transpose_kernel(int N, int pitch, const uint32_t* __restrict__ mask,
                                                        uint32_t* __restrict__ maskT, int* __restrict__ in_count) {
    transpose_task(N, pitch, mask, maskT, in_count, ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32);
}

__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ count, int* __restrict__ row, int N) {
    scan_rows(count, row, N);
}

template <int KIND, int D, bool INCOMING>
__global__ void __launch_bounds__(kFillWarps * 32) fill_kernel(SpaceArgs s, const float* __restrict__ X,
                                                               const uint32_t* __restrict__ M,
                                                               const int* __restrict__ row, int* __restrict__ col,
                                                               float* __restrict__ cost, float* __restrict__ tau,
                                                               const int* __restrict__ out_row,
                                                               const int* __restrict__ out_col,
                                                               const float* __restrict__ out_cost,
                                                               const float* __restrict__ out_tau) {
    fill_row<KIND, D, INCOMING>(s, X, M, row, col, cost, tau, out_row, out_col, out_cost, out_tau,
                                blockIdx.x * kFillWarps + (threadIdx.x >> 5));
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
                   float* tau, bool incoming, const int* orow, const int* ocol, const float* ocost,
                   const float* otau, cudaStream_t st) {
    const int blocks = (s.N + kFillWarps - 1) / kFillWarps;
    if (incoming)
        fill_kernel<KIND, D, true><<<blocks, kFillWarps * 32, 0, st>>>(s, X, M, row, col, cost, tau, orow, ocol,
                                                                        ocost, otau);
    else
        fill_kernel<KIND, D, false><<<blocks, kFillWarps * 32, 0, st>>>(s, X, M, row, col, cost, tau, orow, ocol,
                                                                         ocost, otau);
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

cudaError_t launch_append(const SpaceArgs& s, BoxArgs b, const float* src, int src_pitch, int first, int count,
                          float* X, uint8_t* g, int* f, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((count + 127) / 128);
    if (s.kind == GMT_COST_DI) append_kernel<6, 3><<<blocks, 128, 0, st>>>(s, b, src, src_pitch, first, count, X, g, f);
    else if (s.d == 2) append_kernel<2, 2><<<blocks, 128, 0, st>>>(s, b, src, src_pitch, first, count, X, g, f);
    else if (s.d == 3) append_kernel<3, 3><<<blocks, 128, 0, st>>>(s, b, src, src_pitch, first, count, X, g, f);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_pair_mask(const SpaceArgs& s, const float* X, uint32_t* mask, int* cnt, cudaStream_t st) {
    if (s.kind == GMT_COST_DI) {
        const int W = (s.N + 31) / 32;
        dim3 grid((s.N + kDIRows - 1) / kDIRows, (W + kDIWords - 1) / kDIWords);
        pair_mask_di_kernel<<<grid, kDIRows, 0, st>>>(s, X, mask, cnt);
        return cudaGetLastError();
    }
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
                        float* cost, float* tau, bool incoming, const int* orow, const int* ocol,
                        const float* ocost, const float* otau, cudaStream_t st) {
    if (s.kind == GMT_COST_DI)
        return fill_t<GMT_COST_DI, 6>(s, X, M, row, col, cost, tau, incoming, orow, ocol, ocost, otau, st);
    GMT_EUCLID_DIMS(fill_t, s, X, M, row, col, cost, tau, incoming, orow, ocol, ocost, otau, st)
}

}  // namespace gmtk
