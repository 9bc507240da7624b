// SampleFree and r-disk neighbour graph construction (Section III-B; the
// precomputation of Section V-A), as CUDA kernels for sm_103a.
//
//   sample_kernel     sixteen lanes per node: Philox4x32-10 rejection sampling,
//                     four attempts at once, each attempt's box tests shared
//                     out over four lanes, the first accepted one kept
//   halton_kernel     one block: the free Halton points in order
//   halton_head_kernel + halton_free_kernel  the same split: nodes 0 and 1
//                     in one block, the free points over many blocks (chunks
//                     in ticket order, running totals by look-back)
//   pair_mask_kernel  all ordered pairs (i, j): bit j of row i is set iff
//                     c(i, j) < r; rows staged through shared memory; the bit
//                     matrix is word-major (word w of every row contiguous) so
//                     that each warp writes 32 consecutive rows' words
//   scan_kernel       exclusive prefix sum of the per-row counts -> row_ptr
//   pair_mask_di_kernel  the same for the double integrator: three
//                     conservative tests of increasing cost, then the exact
//                     root procedure, with per-warp compaction between stages;
//                     it also writes the transposed words and in-row counts
//   pair_mask_dubins_kernel  the same for the Dubins airplane: distance
//                     prefilter, then the shortest-word cost from a queue;
//                     it also writes the transposed words and in-row counts
//   scan2_kernel      both directions' row offsets (one block each); the
//                     edge count and sampling flags straight to host memory
//   fill_list_kernel  double integrator, Dubins airplane: the edges the pair
//                     filter listed with their costs (and arrival times or
//                     words), placed in both CSRs by rank (word prefixes
//                     from scan2_kernel's extra blocks)
//   fill_kernel       persistent blocks, eight rows at a time: each warp
//                     gathers a row's columns (prefix over its words) into a
//                     shared-memory list, then the block shares out the eight
//                     rows' edges (two per thread for the double integrator);
//                     out- and in-rows in one launch
#include <atomic>
#include <cstdio>

#include "graph_body.cuh"

namespace gmtk {

// ------------------------------------------------------------------ kernels
constexpr int kSampleThreads = 128;
constexpr int kSampleLanes = 4;     // lanes per attempt: its box tests are shared out
constexpr int kSampleParallel = 4;  // attempts of one node at once
constexpr int kSampleGroup = kSampleLanes * kSampleParallel;  // lanes per node

// Boxes are staged in shared memory when `staged` (2 * count * DP floats): the
// rejection loop then tests them without a global-memory round trip per box.
template <int D, int DP>
__global__ void __launch_bounds__(kSampleThreads) sample_kernel(SpaceArgs s, BoxArgs boxes, BoxGridArgs grid,
                                                                float* __restrict__ X, uint8_t* __restrict__ is_goal,
                                                                int* __restrict__ flags, int staged) {
    extern __shared__ float sbox[];
    if (staged) {
        for (int t = threadIdx.x; t < boxes.count * DP; t += blockDim.x) {
            sbox[t] = boxes.lo[t];
            sbox[boxes.count * DP + t] = boxes.hi[t];
        }
        __syncthreads();
        boxes.lo = sbox;
        boxes.hi = sbox + boxes.count * DP;
    }
    sample_node_group<D, DP, kSampleLanes, kSampleParallel>(s, boxes, grid, X, is_goal, flags,
                                           (int)((blockIdx.x * blockDim.x + threadIdx.x) / kSampleGroup));
}

template <int D, int DP>
__global__ void __launch_bounds__(kHaltonThreads) halton_kernel(SpaceArgs s, BoxArgs boxes, BoxGridArgs grid,
                                                                float* __restrict__ X, uint8_t* __restrict__ is_goal,
                                                                int* __restrict__ flags) {
    halton_sample_block<D, DP>(s, boxes, grid, X, is_goal, flags);
}

template <int D, int DP>
__global__ void __launch_bounds__(kHaltonThreads) halton_head_kernel(SpaceArgs s, BoxArgs boxes, BoxGridArgs grid,
                                                                     float* __restrict__ X,
                                                                     uint8_t* __restrict__ is_goal,
                                                                     int* __restrict__ flags) {
    halton_head_block<D, DP>(s, boxes, grid, X, is_goal, flags);
}

// Nodes 2..n_sampled-1 of the Halton SampleFree: the free points in the order
// of k.  A block takes chunk c (points 1 + c*kHaltonChunk ..) from the ticket,
// counts its free points, publishes the count (flag 1), adds the counts or the
// running total (flag 2) of the chunks before it, walking back until one has a
// running total, and publishes its own; its free points then go to nodes
// 2 + (total before it) + (rank within the chunk).  Chunks are taken in ticket
// order by running blocks, so every chunk a block waits on is held by a
// running block; the first chunk whose total reaches the count stops the rest
// (a chunk after it that finds a predecessor unpublished gives up once it sees
// the stop).  Every wait is bounded (kSampleTimeout).
constexpr long long kHaltonSpinLimit = 1ll << 22;

template <int D, int DP>
__global__ void __launch_bounds__(kHaltonChunk) halton_free_kernel(SpaceArgs s, BoxArgs boxes, BoxGridArgs grid,
                                                                   int* __restrict__ scratch,
                                                                   float* __restrict__ X,
                                                                   uint8_t* __restrict__ is_goal,
                                                                   int* __restrict__ flags) {
    __shared__ int s_chunk, s_quit, s_before, s_go;
    __shared__ int s_warp[kHaltonChunk / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int* ticket = scratch;
    int* stop = scratch + 1;
    unsigned long long* status = reinterpret_cast<unsigned long long*>(scratch + 4);
    const long long need = (long long)s.n_sampled - 2;
    const long long nchunks = (s.halton_cap + kHaltonChunk - 1) / kHaltonChunk;
    constexpr unsigned long long kAgg = 1ull << 62, kInc = 2ull << 62, kVal = (1ull << 62) - 1;
    for (;;) {
        if (tid == 0) {
            s_chunk = atomicAdd(ticket, 1);
            s_quit = s_chunk >= nchunks || *(volatile int*)stop < s_chunk;
        }
        __syncthreads();
        const int c = s_chunk;
        if (s_quit) break;  // the same decision for the whole block
        const long long k = 1 + (long long)c * kHaltonChunk + tid;
        float x[D];
        const bool ok = k <= s.halton_cap && halton_free_point<D, DP>(s, boxes, grid, k, x);
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        if (tid == 0) {
            int count = 0;
            for (int w = 0; w < kHaltonChunk / 32; ++w) count += s_warp[w];
            long long before = 0;
            int go = 1;
            if (c > 0) {
                __threadfence();
                atomicExch(&status[c], kAgg | (unsigned long long)count);
                long long spins = 0;
                for (int j = c - 1; j >= 0;) {
                    const unsigned long long v = atomicAdd(&status[j], 0ull);
                    if ((v >> 62) == 0) {  // not published yet
                        if (*(volatile int*)stop < c) { go = 0; break; }
                        if (++spins > kHaltonSpinLimit) { atomicOr(flags, kSampleTimeout); go = 0; break; }
                        continue;
                    }
                    before += (long long)(v & kVal);
                    if ((v >> 62) == 2) break;
                    --j;
                }
            }
            if (go) {
                const long long total = before + count;
                __threadfence();
                atomicExch(&status[c], kInc | (unsigned long long)total);
                if (total >= need) atomicMin(stop, c);
                else if (c == nchunks - 1) atomicOr(flags, kSampleExhausted);
            }
            s_before = (int)before;
            s_go = go;
        }
        __syncthreads();
        if (s_go && ok) {
            int rank = __popc(m & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w) rank += s_warp[w];
            const long long v = 2 + (long long)s_before + rank;
            if (v < s.n_sampled) {
#pragma unroll
                for (int a = 0; a < D; ++a) X[(size_t)a * s.pitch + v] = x[a];
                is_goal[v] = in_goal_ball(x, s.gd, s.gc, s.grho) ? 1 : 0;
            }
        }
        __syncthreads();
    }
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
                                                              int* __restrict__ out_count,
                                                              int* __restrict__ tile_cnt) {
    mask_tile<KIND, D>(s, X, mask, out_count, blockIdx.x, blockIdx.y, tile_cnt);
}

__global__ void __launch_bounds__(256) tile_prefix_kernel(int N, int pitch, int nb, int* __restrict__ tile_cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) tile_prefix_row(tile_cnt, pitch, nb, i);
}

template <int D>
__global__ void __launch_bounds__(kMaskRows) fill_tile_kernel(SpaceArgs s, const float* __restrict__ X,
                                                              const uint32_t* __restrict__ mask,
                                                              const int* __restrict__ row,
                                                              const int* __restrict__ tile_pre,
                                                              int* __restrict__ col, float* __restrict__ cost,
                                                              long long cap) {
    if (cap > 0 && (long long)__ldg(&row[s.N]) > cap) return;  // uniform: the caller rebuilds
    fill_tile_euclid<D>(s, X, mask, row, tile_pre, col, cost, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(kDIRows, 8) pair_mask_di_kernel(SpaceArgs s, const float* __restrict__ X,
                                                              uint32_t* __restrict__ mask,
                                                              int* __restrict__ out_count,
                                                              uint32_t* __restrict__ maskT,
                                                              int* __restrict__ in_count, int4* __restrict__ elist,
                                                              int* __restrict__ elist_n, int elist_cap) {
    mask_di_tile(s, X, mask, out_count, blockIdx.x, blockIdx.y, maskT, in_count, elist, elist_n, elist_cap);
}

__global__ void __launch_bounds__(kDubRows) pair_mask_dubins_kernel(SpaceArgs s, const float* __restrict__ X,
                                                                  uint32_t* __restrict__ mask,
                                                                  int* __restrict__ out_count,
                                                                  uint32_t* __restrict__ maskT,
                                                                  int* __restrict__ in_count,
                                                                  int4* __restrict__ elist,
                                                                  float4* __restrict__ epath,
                                                                  int* __restrict__ elist_n, int elist_cap) {
    mask_dubins_tile(s, X, mask, out_count, blockIdx.x, blockIdx.y, maskT, in_count, elist, epath, elist_n,
                     elist_cap);
}

__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ count, int* __restrict__ row, int N) {
    scan_rows(count, row, N);
}

// Block 0 scans the out-row counts and, when host_out is given (host memory
// mapped into the device), stores there the build's first two flags (written
// by the kernels before this one) and the edge count, so that the host needs
// no copy; block 1, if count1 is given, scans the in-row counts.  The blocks
// after them, if launched, write the word prefixes of m0 into pre0 and of m1
// into pre1, 32 rows per block (m0's row blocks first).
__global__ void __launch_bounds__(1024) scan2_kernel(const int* __restrict__ count0, int* __restrict__ row0,
                                                     const int* __restrict__ count1, int* __restrict__ row1, int N,
                                                     const int* __restrict__ flags, int* __restrict__ host_out,
                                                     const uint32_t* __restrict__ m0, int* __restrict__ pre0,
                                                     const uint32_t* __restrict__ m1, int* __restrict__ pre1,
                                                     int pitch) {
    const int nscan = count1 ? 2 : 1;
    if ((int)blockIdx.x >= nscan) {
        const int tb = (int)blockIdx.x - nscan, rb = (N + 31) / 32;
        if (tb < rb) word_prefix_block(m0, pre0, N, pitch, 32 * tb);
        else if (m1 && tb < 2 * rb) word_prefix_block(m1, pre1, N, pitch, 32 * (tb - rb));
        return;
    }
    if (blockIdx.x == 0) {
        const int total = scan_rows(count0, row0, N);
        if (threadIdx.x == 0 && host_out) {
            host_out[0] = __ldcg(&flags[0]);
            host_out[1] = __ldcg(&flags[1]);
            host_out[2] = total;
        }
    } else {
        scan_rows(count1, row1, N);
    }
}

// Directed costs: the edges the pair filter listed (with cost and arrival
// time, or shortest word), placed in the out- and in-CSR by their ranks
// (place_listed_edge).  Writes nothing when the edge count exceeds the
// arrays' capacity (cap > 0: the caller rebuilds) or the list's.
template <int KIND>
__global__ void __launch_bounds__(256) fill_list_kernel(int N, int pitch, const int4* __restrict__ elist,
                                                        const float4* __restrict__ epath, int list_cap, FillDir out,
                                                        FillDir in, const int* __restrict__ pre_out,
                                                        const int* __restrict__ pre_in) {
    const int E = __ldg(&out.row[N]);
    if ((out.cap > 0 && (long long)E > out.cap) || E > list_cap || __ldg(&in.row[N]) != E) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < E; t += gridDim.x * blockDim.x)
        place_listed_edge<KIND>(pitch, __ldg(&elist[t]), KIND == GMT_COST_DUBINS ? epath + t : nullptr, out, in,
                                pre_out, pre_in);
}

// Persistent blocks take groups of kFillWarps rows from a ticket counter
// (zeroed with the build's flags): the out-rows' groups, then the in-rows'
// (double integrator, Dubins airplane).  A direction whose edge count exceeds
// its arrays' capacity writes nothing (the caller rebuilds).
template <int KIND, int D>
__global__ void __launch_bounds__(kFillWarps * 32, 4) fill_kernel(SpaceArgs s, const float* __restrict__ X, FillDir out,
                                                               FillDir in, int* __restrict__ ticket) {
    __shared__ FillShared sh;
    const int groups = (s.N + kFillWarps - 1) / kFillWarps;
    const int ngroups = in.mask ? 2 * groups : groups;
    const bool out_ok = !(out.cap > 0 && (long long)__ldg(&out.row[s.N]) > out.cap);
    const bool in_ok = in.mask && !(in.cap > 0 && (long long)__ldg(&in.row[s.N]) > in.cap);
    for (;;) {
        if (threadIdx.x == 0) sh.group = atomicAdd(ticket, 1);
        __syncthreads();
        const int gi = sh.group;
        __syncthreads();  // every thread has read the ticket before thread 0 takes the next
        if (gi >= ngroups) break;
        if (gi < groups) {
            if (out_ok) fill_group<KIND, D, false>(s, X, out, gi * kFillWarps, sh);
        } else if (in_ok) {
            fill_group<KIND, D, true>(s, X, in, (gi - groups) * kFillWarps, sh);
        }
    }
}

// ------------------------------------------------------------------ launchers
namespace {
template <int D, int DP>
cudaError_t sample_t(const SpaceArgs& s, BoxArgs b, const BoxGridArgs& grid, void* scratch, float* X, uint8_t* g,
                     int* f, cudaStream_t st) {
    if (s.sampler == GMT_SAMPLER_HALTON) {
        if (!scratch) {
            halton_kernel<D, DP><<<1, kHaltonThreads, 0, st>>>(s, b, grid, X, g, f);
            return cudaGetLastError();
        }
        halton_head_kernel<D, DP><<<1, kHaltonThreads, 0, st>>>(s, b, grid, X, g, f);
        const long long need = (long long)s.n_sampled - 2;
        if (need <= 0) return cudaGetLastError();
        // about twice the chunks the nodes need when most points are free;
        // blocks loop for more chunks when they are not
        const long long nchunks = (s.halton_cap + kHaltonChunk - 1) / kHaltonChunk;
        long long blocks = 2 * ((need + kHaltonChunk - 1) / kHaltonChunk) + 8;
        if (blocks > nchunks) blocks = nchunks;
        if (blocks > 1024) blocks = 1024;
        halton_free_kernel<D, DP><<<(unsigned)blocks, kHaltonChunk, 0, st>>>(s, b, grid, (int*)scratch, X, g, f);
        return cudaGetLastError();
    }
    const int staged = b.count > 0 && b.count <= 4096 / DP;
    const size_t smem = staged ? (size_t)2 * b.count * DP * sizeof(float) : 0;
    const long long threads = (long long)s.N * kSampleGroup;
    sample_kernel<D, DP><<<(unsigned)((threads + kSampleThreads - 1) / kSampleThreads), kSampleThreads, smem, st>>>(
        s, b, grid, X, g, f, staged);
    return cudaGetLastError();
}
template <int KIND, int D>
cudaError_t mask_t(const SpaceArgs& s, const float* X, uint32_t* mask, int* cnt, int* tile_cnt, cudaStream_t st) {
    const int W = (s.N + 31) / 32, nb = (W + kMaskWords - 1) / kMaskWords;
    dim3 grid((s.N + kMaskRows - 1) / kMaskRows, nb);
    pair_mask_kernel<KIND, D><<<grid, kMaskRows, 0, st>>>(s, X, mask, cnt, tile_cnt);
    // the per-tile counts become prefixes here, so the fill reads them only
    // (and a fill run again on the same mask writes the same CSR)
    if (tile_cnt) tile_prefix_kernel<<<(s.N + 255) / 256, 256, 0, st>>>(s.N, s.pitch, nb, tile_cnt);
    return cudaGetLastError();
}
template <int D>
cudaError_t fill_tiles_t(const SpaceArgs& s, const float* X, const FillDir& out, int* tile_cnt, cudaStream_t st) {
    const int W = (s.N + 31) / 32, nb = (W + kMaskWords - 1) / kMaskWords;
    dim3 grid((s.N + kMaskRows - 1) / kMaskRows, nb);
    fill_tile_kernel<D><<<grid, kMaskRows, 0, st>>>(s, X, out.mask, out.row, tile_cnt, out.col, out.cost, out.cap);
    return cudaGetLastError();
}
template <int KIND, int D>
cudaError_t fill_t(const SpaceArgs& s, const float* X, const FillDir& out, const FillDir& in, int* ticket,
                   cudaStream_t st) {
    // as many blocks as fit on the GPU at once (queried once per instantiation;
    // any count is correct, the blocks take groups until none is left)
    static std::atomic<int> resident_cache{0};
    int resident = resident_cache.load(std::memory_order_relaxed);
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fill_kernel<KIND, D>, kFillWarps * 32, 0);
        if (e != cudaSuccess) return e;
        resident = sms * (per_sm > 0 ? per_sm : 1);
        resident_cache.store(resident, std::memory_order_relaxed);
    }
    const long long groups = (long long)((s.N + kFillWarps - 1) / kFillWarps) * (in.mask ? 2 : 1);
    const int blocks = (int)(groups < resident ? groups : resident);
    fill_kernel<KIND, D><<<blocks, kFillWarps * 32, 0, st>>>(s, X, out, in, ticket);
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

cudaError_t launch_sample(const SpaceArgs& s, BoxArgs b, const BoxGridArgs& grid, void* scratch, float* X,
                          uint8_t* g, int* f, cudaStream_t st) {
    if (s.kind == GMT_COST_DI) return sample_t<6, 3>(s, b, grid, scratch, X, g, f, st);
    if (s.kind == GMT_COST_DUBINS) return sample_t<4, 3>(s, b, grid, scratch, X, g, f, st);
    switch (s.d) {
        case 2: return sample_t<2, 2>(s, b, grid, scratch, X, g, f, st);
        case 3: return sample_t<3, 3>(s, b, grid, scratch, X, g, f, st);
        case 4: return sample_t<4, 4>(s, b, grid, scratch, X, g, f, st);
        case 5: return sample_t<5, 5>(s, b, grid, scratch, X, g, f, st);
        case 6: return sample_t<6, 6>(s, b, grid, scratch, X, g, f, st);
        case 7: return sample_t<7, 7>(s, b, grid, scratch, X, g, f, st);
        case 8: return sample_t<8, 8>(s, b, grid, scratch, X, g, f, st);
        case 9: return sample_t<9, 9>(s, b, grid, scratch, X, g, f, st);
        case 10: return sample_t<10, 10>(s, b, grid, scratch, X, g, f, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_append(const SpaceArgs& s, BoxArgs b, const float* src, int src_pitch, int first, int count,
                          float* X, uint8_t* g, int* f, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((count + 127) / 128);
    if (s.kind == GMT_COST_DI) append_kernel<6, 3><<<blocks, 128, 0, st>>>(s, b, src, src_pitch, first, count, X, g, f);
    else if (s.kind == GMT_COST_DUBINS)
        append_kernel<4, 3><<<blocks, 128, 0, st>>>(s, b, src, src_pitch, first, count, X, g, f);
    else if (s.d == 2) append_kernel<2, 2><<<blocks, 128, 0, st>>>(s, b, src, src_pitch, first, count, X, g, f);
    else if (s.d == 3) append_kernel<3, 3><<<blocks, 128, 0, st>>>(s, b, src, src_pitch, first, count, X, g, f);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_pair_mask(const SpaceArgs& s, const float* X, uint32_t* mask, int* cnt, uint32_t* maskT,
                             int* in_count, cudaStream_t st, int* tile_cnt, int4* elist, int* elist_n,
                             int elist_cap, float4* epath) {
    if (s.kind == GMT_COST_DI) {
        const int W = (s.N + 31) / 32;
        dim3 grid((s.N + kDIRows - 1) / kDIRows, (W + kDIWords - 1) / kDIWords);
        pair_mask_di_kernel<<<grid, kDIRows, 0, st>>>(s, X, mask, cnt, maskT, in_count, elist, elist_n, elist_cap);
        return cudaGetLastError();
    }
    if (s.kind == GMT_COST_DUBINS) {
        const int W = (s.N + 31) / 32;
        dim3 grid((s.N + kDubRows - 1) / kDubRows, (W + kDubWords - 1) / kDubWords);
        pair_mask_dubins_kernel<<<grid, kDubRows, 0, st>>>(s, X, mask, cnt, maskT, in_count, epath ? elist : nullptr,
                                                           epath, elist_n, elist_cap);
        return cudaGetLastError();
    }
    GMT_EUCLID_DIMS(mask_t, s, X, mask, cnt, s.d >= 2 && s.d <= 4 ? tile_cnt : nullptr, st)
}

int fill_tiles_per_row(int N) {
    const int W = (N + 31) / 32;
    return (W + kMaskWords - 1) / kMaskWords;
}

cudaError_t launch_fill_tiles(const SpaceArgs& s, const float* X, const FillDir& out, int* tile_cnt,
                              cudaStream_t st) {
    if (s.d == 2) return fill_tiles_t<2>(s, X, out, tile_cnt, st);
    if (s.d == 3) return fill_tiles_t<3>(s, X, out, tile_cnt, st);
    if (s.d == 4) return fill_tiles_t<4>(s, X, out, tile_cnt, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_scan(const int* count, int* row, int N, cudaStream_t st) {
    scan_kernel<<<1, 1024, 0, st>>>(count, row, N);
    return cudaGetLastError();
}

cudaError_t launch_scan2(const int* count0, int* row0, const int* count1, int* row1, int N, const int* flags,
                         int* host_out, cudaStream_t st, const uint32_t* m0, int* pre0, const uint32_t* m1,
                         int* pre1, int pitch) {
    const int nscan = count1 ? 2 : 1;
    const int ntab = m0 && pre0 ? (m1 && pre1 ? 2 : 1) * ((N + 31) / 32) : 0;  // 32 rows per block
    scan2_kernel<<<nscan + ntab, 1024, 0, st>>>(count0, row0, count1, row1, N, flags, host_out, m0, pre0,
                                                m1 && pre1 ? m1 : nullptr, pre1, pitch);
    return cudaGetLastError();
}

cudaError_t launch_fill_list(const SpaceArgs& s, const int4* elist, const float4* epath, int list_cap,
                             const FillDir& out, const FillDir& in, const int* pre_out, const int* pre_in,
                             cudaStream_t st) {
    long long blocks = ((long long)list_cap + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    if (s.kind == GMT_COST_DI)
        fill_list_kernel<GMT_COST_DI>
            <<<(unsigned)blocks, 256, 0, st>>>(s.N, s.pitch, elist, nullptr, list_cap, out, in, pre_out, pre_in);
    else if (s.kind == GMT_COST_DUBINS && epath && in.path)
        fill_list_kernel<GMT_COST_DUBINS>
            <<<(unsigned)blocks, 256, 0, st>>>(s.N, s.pitch, elist, epath, list_cap, out, in, pre_out, pre_in);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_fill(const SpaceArgs& s, const float* X, const FillDir& out, const FillDir& in, int* ticket,
                        cudaStream_t st) {
    if (s.kind == GMT_COST_DI) return fill_t<GMT_COST_DI, 6>(s, X, out, in, ticket, st);
    if (s.kind == GMT_COST_DUBINS) return fill_t<GMT_COST_DUBINS, 4>(s, X, out, in, ticket, st);
    GMT_EUCLID_DIMS(fill_t, s, X, out, in, ticket, st)
}

}  // namespace gmtk
