// Learned sampling proposal (an extension of the paper's uniform SampleFree):
// an MLP maps a voxelised obstacle map plus start and goal to logits over a
// coarse grid of cells; samples are drawn from the softmax over cells, then
// uniformly inside the chosen cell, and rejected if they collide.
//
//   X  [B, G^3]  voxel occupancy (BF16 0/1; voxel centres tested against the boxes)
//   H1 = relu(X W1^T + b1)              [B, H]        (GEMM, split-K over G^3)
//   H2 = relu(H1 W2^T + b2)             [B, H]
//   Z  = [H2, start(3), goal(3), 0..]   [B, H + 16]
//   logits = Z W3^T + b3                [B, C^3]
// Training: softmax cross-entropy against a target distribution over cells,
// backward through the same BF16 tensor-core GEMM with FP32 accumulation
// (dW = dY^T X computed as GEMMs of transposed BF16 copies), AdamW on FP32
// master weights, BF16 copies refreshed after every step.
#include <cmath>
#include <cstdio>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

using namespace gmtk;
typedef __nv_bfloat16 bf16;

namespace {

// ------------------------------------------------------------------ kernels
struct EnvBoxes {
    int count;
    const float* lo;
    const float* hi;
};

// X[b, (i G + j) G + k] = 1 if the centre of voxel (i, j, k) lies in a box of env b.
constexpr int kVoxBoxes = 256;  // boxes staged in shared memory per pass
constexpr int kVoxRows = 256;   // voxel rows (i, j) per block

// Block (x, b): rows (i, j) of environment b's voxel grid, one thread per row
// of G voxels along k; its boxes pass through shared memory.  A box is tested
// against the row's centre in x and y once, and only then against the G
// centres in z, so a voxel is occupied exactly when its centre lies in a box
// (the same comparisons as testing every voxel against every box).
__global__ void __launch_bounds__(kVoxRows) voxelize_kernel(const EnvBoxes* __restrict__ envs, int G,
                                                            bf16* __restrict__ X) {
    __shared__ float slo[kVoxBoxes * 3], shi[kVoxBoxes * 3];
    __shared__ float pz[64];
    const int b = blockIdx.y;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = row / G, j = row % G;
    const float px = ((float)i + 0.5f) / (float)G, py = ((float)j + 0.5f) / (float)G;
    if (threadIdx.x < G) pz[threadIdx.x] = ((float)threadIdx.x + 0.5f) / (float)G;
    const EnvBoxes e = envs[b];
    unsigned long long occ = 0ull;
    for (int b0 = 0; b0 < e.count; b0 += kVoxBoxes) {
        const int nb = min(kVoxBoxes, e.count - b0);
        __syncthreads();  // the previous pass's boxes are no longer read
        for (int t = threadIdx.x; t < nb * 3; t += blockDim.x) {
            slo[t] = e.lo[(size_t)b0 * 3 + t];
            shi[t] = e.hi[(size_t)b0 * 3 + t];
        }
        __syncthreads();
        for (int q = 0; q < nb; ++q) {
            if (slo[3 * q] <= px && px <= shi[3 * q] && slo[3 * q + 1] <= py && py <= shi[3 * q + 1]) {
                const float zl = slo[3 * q + 2], zh = shi[3 * q + 2];
                for (int k = 0; k < G; ++k)
                    if (zl <= pz[k] && pz[k] <= zh) occ |= 1ull << k;
            }
        }
    }
    if (row >= G * G) return;
    bf16* out = X + (size_t)b * G * G * G + (size_t)row * G;
    const unsigned short one = 0x3F80u;  // BF16 1.0
    if (G % 8 == 0 && ((uintptr_t)out & 15u) == 0) {
        for (int k0 = 0; k0 < G; k0 += 8) {
            unsigned w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const unsigned lo = (occ >> (k0 + 2 * h)) & 1ull ? one : 0u;
                const unsigned hi = (occ >> (k0 + 2 * h + 1)) & 1ull ? one : 0u;
                w[h] = lo | (hi << 16);
            }
            *reinterpret_cast<uint4*>(out + k0) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        for (int k = 0; k < G; ++k) out[k] = __float2bfloat16_rn((occ >> k) & 1ull ? 1.0f : 0.0f);
    }
}

// Z = [H2, start/goal (6), zeros] in BF16.
__global__ void concat_kernel(const bf16* __restrict__ H2, const float* __restrict__ sg, int B, int H, int Dz,
                              bf16* __restrict__ Z) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * Dz) return;
    const int b = t / Dz, c = t % Dz;
    bf16 v = __float2bfloat16_rn(0.0f);
    if (c < H) v = H2[(size_t)b * H + c];
    else if (c < H + 6) v = __float2bfloat16_rn(sg[b * 6 + (c - H)]);
    Z[t] = v;
}

// [R, C] -> [C, R] through 32x32 shared-memory tiles.
__global__ void transpose_bf16_kernel(const bf16* __restrict__ in, int R, int C, bf16* __restrict__ out) {
    __shared__ bf16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[y][threadIdx.x] = in[(size_t)r * C + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * R + r] = tile[threadIdx.x][y];
    }
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ in, long long n, bf16* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = __float2bfloat16_rn(in[t]);
}

// Row-wise softmax cross-entropy: loss_b = -sum_c T_bc log softmax(l_b)_c and
// dlogits = (softmax - T) / B (rounded to BF16 for the backward GEMMs).
__global__ void softmax_xent_kernel(const float* __restrict__ logits, const float* __restrict__ T, int B, int Nc,
                                    bf16* __restrict__ dlog, float* __restrict__ loss) {
    __shared__ float red[32];
    const int b = blockIdx.x;
    const float* l = logits + (size_t)b * Nc;
    const float* t = T + (size_t)b * Nc;
    float mx = -INFINITY;
    for (int c = threadIdx.x; c < Nc; c += blockDim.x) mx = fmaxf(mx, l[c]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        red[0] = v;
    }
    __syncthreads();
    mx = red[0];
    __syncthreads();
    float se = 0.0f;
    for (int c = threadIdx.x; c < Nc; c += blockDim.x) se += expf(l[c] - mx);
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        red[0] = v;
    }
    __syncthreads();
    const float lse = mx + logf(red[0]);
    __syncthreads();
    float lo = 0.0f;
    for (int c = threadIdx.x; c < Nc; c += blockDim.x) {
        const float p = expf(l[c] - lse);
        lo -= t[c] * (l[c] - lse);
        if (dlog) dlog[(size_t)b * Nc + c] = __float2bfloat16_rn((p - t[c]) / (float)B);
    }
    for (int o = 16; o > 0; o >>= 1) lo += __shfl_xor_sync(0xffffffffu, lo, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        loss[b] = s;
    }
}

// dpre = d[:, :H] * (act > 0) in BF16 (d has row stride ld).
__global__ void relu_back_kernel(const float* __restrict__ d, int ld, const bf16* __restrict__ act, int B, int H,
                                 bf16* __restrict__ dpre) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * H) return;
    const int b = t / H, c = t % H;
    const float a = __bfloat162float(act[t]);
    dpre[t] = __float2bfloat16_rn(a > 0.0f ? d[(size_t)b * ld + c] : 0.0f);
}

// g[c] = sum_b d[b, c] (d BF16 [B, N] or FP32).
// Column sums of a BF16 matrix [B][N] in FP32: a block of 32 x 8 threads takes
// 32 columns, each thread a strided eighth of the rows, then the 8 partial
// sums are added in a fixed order (deterministic).
__global__ void __launch_bounds__(256) colsum_bf16_kernel(const bf16* __restrict__ d, int B, int N,
                                                         float* __restrict__ g) {
    __shared__ float part[8][33];
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cx;
    float s = 0.0f;
    if (c < N)
        for (int b = ry; b < B; b += 8) s += __bfloat162float(d[(size_t)b * N + c]);
    part[ry][cx] = s;
    __syncthreads();
    if (ry == 0 && c < N) {
        float t = part[0][cx];
        for (int k = 1; k < 8; ++k) t += part[k][cx];
        g[c] = t;
    }
}

// AdamW (decoupled weight decay) on FP32 master weights; refreshes the BF16 copy.
__global__ void adamw_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float wd,
                             float c1, float c2, bf16* __restrict__ pb) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.0f - b1) * gt;
    const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    float w = p[t] * (1.0f - lr * wd);
    w -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    p[t] = w;
    if (pb) pb[t] = __float2bfloat16_rn(w);
}

// Deterministic N(0, std^2) initial weights from Philox (Box-Muller).
__global__ void init_normal_kernel(float* __restrict__ p, long long n, float std, uint32_t k0, uint32_t k1,
                                   uint32_t tensor) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const Ctr4 c = philox4x32_10(Ctr4{(uint32_t)t, (uint32_t)(t >> 32), 3u, tensor}, k0, k1);
    const float u1 = ((float)(c.x >> 8) + 1.0f) * 0x1p-24f;
    const float u2 = (float)(c.y >> 8) * 0x1p-24f;
    p[t] = std * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// Normalised histogram over cells^3 of points every `spacing` along a path of
// sample indices (positions are the first three coordinates), plus eps.
// Path histogram in one block: points every `spacing` along the path (each
// segment from its start, m = max(1, ceil(L / spacing)) points at t = k/m,
// then the last node), counted per cell in shared memory (the counts are whole
// numbers, so the order of the additions does not matter), then
// normalised: (count + eps) / (total + eps cells^3).
__global__ void __launch_bounds__(256) path_hist_kernel(const float* __restrict__ X, int pitch,
                                                        const int* __restrict__ path, int len, int cells,
                                                        float spacing, float eps, float* __restrict__ hist) {
    extern __shared__ float h[];
    __shared__ float red[256];
    const int n = cells * cells * cells;
    for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = 0.0f;
    __syncthreads();
    auto cell_of = [&](const float* x) {
        int idx = 0;
        for (int d = 0; d < 3; ++d) {
            int ci = (int)(x[d] * (float)cells);
            ci = min(max(ci, 0), cells - 1);
            idx = idx * cells + ci;
        }
        return idx;
    };
    for (int s = threadIdx.x; s + 1 < len; s += blockDim.x) {
        const int a = path[s], b = path[s + 1];
        float pa[3], pb[3];
        for (int d = 0; d < 3; ++d) { pa[d] = X[(size_t)d * pitch + a]; pb[d] = X[(size_t)d * pitch + b]; }
        const float L = sqrtf((pb[0] - pa[0]) * (pb[0] - pa[0]) + (pb[1] - pa[1]) * (pb[1] - pa[1]) +
                              (pb[2] - pa[2]) * (pb[2] - pa[2]));
        const int m = max(1, (int)ceilf(L / spacing));
        for (int k = 0; k < m; ++k) {
            const float t = (float)k / (float)m;
            float x[3];
            for (int d = 0; d < 3; ++d) x[d] = pa[d] + t * (pb[d] - pa[d]);
            atomicAdd(&h[cell_of(x)], 1.0f);
        }
    }
    if (threadIdx.x == 0 && len >= 1) {
        const int e = path[len - 1];
        float x[3];
        for (int d = 0; d < 3; ++d) x[d] = X[(size_t)d * pitch + e];
        atomicAdd(&h[cell_of(x)], 1.0f);
    }
    __syncthreads();
    // total count: whole numbers below 2^24, exact in any order
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += h[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const float tot = red[0] + eps * (float)n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) hist[i] = (h[i] + eps) / tot;
}

// One environment of a proposal launch: its obstacle boxes, position bounds,
// Philox key and output rows (3 x pitch floats).
struct ProposalEnv {
    int box_count;
    const float* box_lo;
    const float* box_hi;
    float lo[3], hi[3];
    uint32_t k0, k1;
    float* out;
};

// One block per environment (blockIdx.x; its logits are row blockIdx.x of
// `logits`).  Draws `count` samples: a cell from the softmax of the logits
// (inverse CDF, Philox counter (k, attempt, 2, 0)), a uniform point inside it
// (same draw), rejected while it lies in a box; velocity-free 3D positions.
// The CDF is a block-wide scan: each thread sums a contiguous run of cells,
// the run totals are scanned across warps, and each thread writes its run's
// running sums from its offset.
__global__ void __launch_bounds__(1024) proposal_sample_kernel(const float* __restrict__ logits, int Nc, int cells,
                                                               const ProposalEnv* __restrict__ envs, int count,
                                                               int max_attempts, int pitch,
                                                               int* __restrict__ flags) {
    extern __shared__ float cdf[];
    __shared__ float red[32];
    __shared__ float blo[3], bhi[3];
    const ProposalEnv& E = envs[blockIdx.x];
    const float* lg = logits + (size_t)blockIdx.x * Nc;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    if (threadIdx.x < 3) { blo[threadIdx.x] = E.lo[threadIdx.x]; bhi[threadIdx.x] = E.hi[threadIdx.x]; }
    float mx = -INFINITY;
    for (int c = threadIdx.x; c < Nc; c += blockDim.x) mx = fmaxf(mx, lg[c]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = -INFINITY;
        for (int w = 0; w < nw; ++w) v = fmaxf(v, red[w]);
        red[0] = v;
    }
    __syncthreads();
    mx = red[0];
    __syncthreads();  // red is reused by the scan
    // this thread's run of cells [c0, c1)
    const int per = (Nc + (int)blockDim.x - 1) / (int)blockDim.x;
    const int c0 = min(Nc, (int)threadIdx.x * per), c1 = min(Nc, c0 + per);
    float run = 0.0f;
    for (int c = c0; c < c1; ++c) {
        const float v = expf(lg[c] - mx);
        cdf[c] = v;
        run += v;
    }
    float inc = run;  // inclusive scan of the run totals within the warp
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) red[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        float w = lane < nw ? red[lane] : 0.0f;
        for (int o = 1; o < 32; o <<= 1) {
            const float t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) red[lane] = w;
    }
    __syncthreads();
    const float excl = __shfl_up_sync(0xffffffffu, inc, 1);
    float acc = (wid > 0 ? red[wid - 1] : 0.0f) + (lane > 0 ? excl : 0.0f);
    for (int c = c0; c < c1; ++c) {
        acc += cdf[c];
        cdf[c] = acc;
    }
    __syncthreads();
    const float total = cdf[Nc - 1];
    const float w = 1.0f / (float)cells;
    const BoxArgs boxes{E.box_count, E.box_lo, E.box_hi};
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        bool ok = false;
        float p[3] = {0, 0, 0};
        for (int t = 0; t < max_attempts && !ok; ++t) {
            const Ctr4 r = philox4x32_10(Ctr4{(uint32_t)k, (uint32_t)t, 2u, 0u}, E.k0, E.k1);
            const float u = unit_float(r.x) * total;
            int lo_i = 0, hi_i = Nc - 1;
            while (lo_i < hi_i) {
                const int mid = (lo_i + hi_i) >> 1;
                if (cdf[mid] > u) hi_i = mid; else lo_i = mid + 1;
            }
            const int cell = lo_i;
            const int ci[3] = {cell / (cells * cells), (cell / cells) % cells, cell % cells};
            const float uu[3] = {unit_float(r.y), unit_float(r.z), unit_float(r.w)};
            for (int d = 0; d < 3; ++d) {
                const float x01 = ((float)ci[d] + uu[d]) * w;
                p[d] = blo[d] + x01 * (bhi[d] - blo[d]);
            }
            ok = !in_any_box<3>(p, boxes.lo, boxes.hi, boxes.count);
        }
        if (!ok) atomicOr(flags, 1);
        for (int d = 0; d < 3; ++d) E.out[(size_t)d * pitch + k] = p[d];
    }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ===================================================================== model
struct gmt_model {
    int G = 32, H = 512, C = 16, Din = 0, Dz = 0, Nc = 0, maxB = 0;
    long long step = 0;
    uint64_t seed = 0;
    // parameters (FP32 masters), BF16 copies, Adam moments, gradients
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr, *W3 = nullptr, *b3 = nullptr;
    bf16 *W1b = nullptr, *W2b = nullptr, *W2tb = nullptr, *W3b = nullptr, *W3tb = nullptr;
    float* mom[6] = {};
    float* vel[6] = {};
    float *gW1 = nullptr, *gb1 = nullptr, *gW2 = nullptr, *gb2 = nullptr, *gW3 = nullptr, *gb3 = nullptr;
    // activations for up to maxB environments
    bf16 *Xt = nullptr, *H1 = nullptr, *H1t = nullptr, *H2 = nullptr, *Z = nullptr, *Zt = nullptr;
    bf16 *dlog = nullptr, *dlogt = nullptr, *dH2 = nullptr, *dH2t = nullptr, *dH1p = nullptr, *dH1pt = nullptr;
    float *logits = nullptr, *dZ = nullptr, *dH1 = nullptr, *ws = nullptr, *loss = nullptr;
    size_t ws_floats = 0;
    int* err = nullptr;
    // proposal scratch
    bf16* pvox = nullptr;
    float* psg = nullptr;
    EnvBoxes* envs = nullptr;       // grow-only descriptor arrays of proposal calls
    ProposalEnv* penv = nullptr;
    int envs_cap = 0;
    unsigned char* pin = nullptr;   // pinned staging of those descriptors and start/goal
    size_t pin_cap = 0;
    cudaEvent_t pin_ev = nullptr;   // recorded after the copies out of `pin`
    std::vector<void*> owned;

    long long n(int i) const {
        const long long s[6] = {(long long)H * Din, H, (long long)H * H, H, (long long)Nc * Dz, Nc};
        return s[i];
    }
    float* param(int i) { float* p[6] = {W1, b1, W2, b2, W3, b3}; return p[i]; }
    float* grad(int i) { float* p[6] = {gW1, gb1, gW2, gb2, gW3, gb3}; return p[i]; }
    ~gmt_model() {
        for (void* p : owned) cudaFree(p);
        if (envs) cudaFree(envs);
        if (penv) cudaFree(penv);
        if (pin) cudaFreeHost(pin);
        if (pin_ev) cudaEventDestroy(pin_ev);
    }
};

namespace {

template <class T>
cudaError_t mk(gmt_model* m, T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, (count ? count : 1) * sizeof(T));
    if (e == cudaSuccess) m->owned.push_back(*p);
    return e;
}

gmt_status mfail(gmt_status s, const std::string& msg) {
    record_error(msg.c_str());
    return s;
}
gmt_status mcuda(cudaError_t e, const char* what) {
    return mfail(e == cudaErrorMemoryAllocation ? GMT_ERR_OOM : GMT_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}
#define MCUDA(call, what)                               \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return mcuda(e_, what);  \
    } while (0)

cudaError_t transpose(const bf16* in, int R, int C, bf16* out, cudaStream_t st) {
    dim3 grid((C + 31) / 32, (R + 31) / 32);
    transpose_bf16_kernel<<<grid, dim3(32, 8), 0, st>>>(in, R, C, out);
    return cudaGetLastError();
}

// Split-K factor: enough K-slices that the CTAs cover the SMs once (each
// slice at least 4 K-blocks deep).
int splits_for(int M, int N, int K) {
    static std::atomic<int> sms_cached{0};
    int sms = sms_cached.load(std::memory_order_relaxed);
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
        sms_cached.store(sms, std::memory_order_relaxed);
    }
    const int tiles = ((M + 127) / 128) * ((N + 127) / 128);
    const int kb = (K + 63) / 64;
    if (tiles >= sms) return 1;
    int s = sms / tiles;
    if (s > kb / 4) s = kb / 4;
    return s < 1 ? 1 : s;
}

cudaError_t gemm(gmt_model* m, int M, int N, int K, const bf16* A, const bf16* B, int epi, const float* bias,
                 float* C, bf16* Cb, cudaStream_t st) {
    int s = splits_for(M, N, K);
    while (s > 1 && (size_t)s * M * N > m->ws_floats) s /= 2;
    return gemm_bf16_tn(M, N, K, A, B, epi, bias, C, Cb, N, s, m->ws, m->err, st);
}

// Refresh the BF16 copies (and transposed copies) of the weights.
cudaError_t refresh_copies(gmt_model* m, cudaStream_t st) {
    f32_to_bf16_kernel<<<blocks_for(m->n(0), 256), 256, 0, st>>>(m->W1, m->n(0), m->W1b);
    f32_to_bf16_kernel<<<blocks_for(m->n(2), 256), 256, 0, st>>>(m->W2, m->n(2), m->W2b);
    f32_to_bf16_kernel<<<blocks_for(m->n(4), 256), 256, 0, st>>>(m->W3, m->n(4), m->W3b);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = transpose(m->W2b, m->H, m->H, m->W2tb, st);
    if (e == cudaSuccess) e = transpose(m->W3b, m->Nc, m->Dz, m->W3tb, st);
    return e;
}

gmt_status forward(gmt_model* m, int B, const bf16* X, const float* sg, cudaStream_t st) {
    MCUDA(gemm(m, B, m->H, m->Din, X, m->W1b, 1, m->b1, nullptr, m->H1, st), "layer 1 GEMM");
    MCUDA(gemm(m, B, m->H, m->H, m->H1, m->W2b, 1, m->b2, nullptr, m->H2, st), "layer 2 GEMM");
    concat_kernel<<<blocks_for((long long)B * m->Dz, 256), 256, 0, st>>>(m->H2, sg, B, m->H, m->Dz, m->Z);
    MCUDA(cudaGetLastError(), "concat");
    MCUDA(gemm(m, B, m->Nc, m->Dz, m->Z, m->W3b, 2, m->b3, m->logits, nullptr, st), "layer 3 GEMM");
    return GMT_OK;
}

gmt_status backward(gmt_model* m, int B, const bf16* X, const float* target, cudaStream_t st) {
    softmax_xent_kernel<<<B, 256, 0, st>>>(m->logits, target, B, m->Nc, m->dlog, m->loss);
    MCUDA(cudaGetLastError(), "softmax cross-entropy");
    // layer 3
    MCUDA(transpose(m->dlog, B, m->Nc, m->dlogt, st), "transpose");
    MCUDA(transpose(m->Z, B, m->Dz, m->Zt, st), "transpose");
    MCUDA(gemm(m, m->Nc, m->Dz, B, m->dlogt, m->Zt, 0, nullptr, m->gW3, nullptr, st), "dW3 GEMM");
    colsum_bf16_kernel<<<blocks_for(m->Nc, 32), 256, 0, st>>>(m->dlog, B, m->Nc, m->gb3);
    MCUDA(gemm(m, B, m->Dz, m->Nc, m->dlog, m->W3tb, 0, nullptr, m->dZ, nullptr, st), "dZ GEMM");
    // layer 2
    relu_back_kernel<<<blocks_for((long long)B * m->H, 256), 256, 0, st>>>(m->dZ, m->Dz, m->H2, B, m->H, m->dH2);
    MCUDA(cudaGetLastError(), "relu backward");
    MCUDA(transpose(m->dH2, B, m->H, m->dH2t, st), "transpose");
    MCUDA(transpose(m->H1, B, m->H, m->H1t, st), "transpose");
    MCUDA(gemm(m, m->H, m->H, B, m->dH2t, m->H1t, 0, nullptr, m->gW2, nullptr, st), "dW2 GEMM");
    colsum_bf16_kernel<<<blocks_for(m->H, 32), 256, 0, st>>>(m->dH2, B, m->H, m->gb2);
    MCUDA(gemm(m, B, m->H, m->H, m->dH2, m->W2tb, 0, nullptr, m->dH1, nullptr, st), "dH1 GEMM");
    // layer 1
    relu_back_kernel<<<blocks_for((long long)B * m->H, 256), 256, 0, st>>>(m->dH1, m->H, m->H1, B, m->H, m->dH1p);
    MCUDA(cudaGetLastError(), "relu backward");
    MCUDA(transpose(m->dH1p, B, m->H, m->dH1pt, st), "transpose");
    MCUDA(transpose(X, B, m->Din, m->Xt, st), "transpose");
    MCUDA(gemm(m, m->H, m->Din, B, m->dH1pt, m->Xt, 0, nullptr, m->gW1, nullptr, st), "dW1 GEMM");
    colsum_bf16_kernel<<<blocks_for(m->H, 32), 256, 0, st>>>(m->dH1p, B, m->H, m->gb1);
    MCUDA(cudaGetLastError(), "bias gradients");
    return GMT_OK;
}

gmt_status check_err(gmt_model* m, cudaStream_t st) {
    int h = 0;
    MCUDA(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, st), "error flag");
    MCUDA(cudaStreamSynchronize(st), "model step");
    if (h) {
        cudaMemsetAsync(m->err, 0, sizeof(int), st);
        return mfail(GMT_ERR_TIMEOUT, "a tensor-core GEMM wait ran out");
    }
    return GMT_OK;
}

// Proposal draws for B environments: descriptors uploaded once, then per
// chunk of at most maxB environments the voxelisation, one batched forward
// pass and one sampling launch (one block per environment); one host
// synchronisation at the end reads the exhausted-attempts flag.
gmt_status propose_impl(gmt_model* m, int B, const gmt_space* spaces, const gmt_boxes* boxes, const float* sg,
                        int count, const uint64_t* seeds, float* samples, int pitch, gmt_stream stream) {
    if (!m || B < 1 || !spaces || !boxes || !sg || !seeds || !samples || count < 1 || pitch < count)
        return mfail(GMT_ERR_INVALID, "bad proposal arguments");
    const size_t smem = (size_t)m->Nc * sizeof(float);  // at most 32^3 cells: 128 KB
    static std::atomic<bool> attr_set{false};
    if (smem > 48 * 1024 && !attr_set.load(std::memory_order_relaxed)) {
        MCUDA(cudaFuncSetAttribute(proposal_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   128 * 1024),
              "proposal kernel attribute");
        attr_set.store(true, std::memory_order_relaxed);
    }
    // pinned staging: [B] EnvBoxes, [B] ProposalEnv, [B][6] start/goal
    const size_t eb_bytes = (size_t)B * sizeof(EnvBoxes), pe_bytes = (size_t)B * sizeof(ProposalEnv);
    const size_t pe_off = (eb_bytes + 15) / 16 * 16, sg_off = pe_off + (pe_bytes + 15) / 16 * 16;
    const size_t need = sg_off + (size_t)B * 6 * sizeof(float);
    if (!m->pin_ev) MCUDA(cudaEventCreateWithFlags(&m->pin_ev, cudaEventDisableTiming), "proposal event");
    MCUDA(cudaEventSynchronize(m->pin_ev), "proposal staging");  // earlier copies out of `pin` are done
    if (m->pin_cap < need) {
        if (m->pin) cudaFreeHost(m->pin);
        m->pin = nullptr;
        m->pin_cap = 0;
        MCUDA(cudaMallocHost((void**)&m->pin, need), "proposal staging");
        m->pin_cap = need;
    }
    EnvBoxes* eb = (EnvBoxes*)m->pin;
    ProposalEnv* pe = (ProposalEnv*)(m->pin + pe_off);
    float* hsg = (float*)(m->pin + sg_off);
    std::memcpy(hsg, sg, (size_t)B * 6 * sizeof(float));
    for (int b = 0; b < B; ++b) {
        const gmt_space& sp = spaces[b];
        if (sp.kind != GMT_COST_EUCLID || sp.dim != 3)
            return mfail(GMT_ERR_INVALID, "the learned proposal supports 3D geometric spaces");
        if (boxes[b].count < 0 || (boxes[b].count > 0 && (!boxes[b].lo || !boxes[b].hi)))
            return mfail(GMT_ERR_INVALID, "bad box arrays");
        eb[b] = EnvBoxes{boxes[b].count, boxes[b].lo, boxes[b].hi};
        ProposalEnv& e = pe[b];
        e.box_count = boxes[b].count; e.box_lo = boxes[b].lo; e.box_hi = boxes[b].hi;
        for (int a = 0; a < 3; ++a) { e.lo[a] = sp.lo[a]; e.hi[a] = sp.hi[a]; }
        e.k0 = (uint32_t)(seeds[b] & 0xffffffffu);
        e.k1 = (uint32_t)(seeds[b] >> 32);
        e.out = samples + (size_t)b * 3 * pitch;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (m->envs_cap < B) {
        MCUDA(cudaStreamSynchronize(st), "proposal descriptors");  // earlier calls may still read them
        if (m->envs) cudaFree(m->envs);
        if (m->penv) cudaFree(m->penv);
        m->envs = nullptr; m->penv = nullptr; m->envs_cap = 0;
        MCUDA(cudaMalloc((void**)&m->envs, (size_t)B * sizeof(EnvBoxes)), "proposal descriptors");
        MCUDA(cudaMalloc((void**)&m->penv, (size_t)B * sizeof(ProposalEnv)), "proposal descriptors");
        m->envs_cap = B;
    }
    MCUDA(cudaMemcpyAsync(m->envs, eb, eb_bytes, cudaMemcpyHostToDevice, st), "proposal descriptors");
    MCUDA(cudaMemcpyAsync(m->penv, pe, pe_bytes, cudaMemcpyHostToDevice, st), "proposal descriptors");
    for (int b0 = 0; b0 < B; b0 += m->maxB) {
        const int nb = std::min(m->maxB, B - b0);
        MCUDA(cudaMemcpyAsync(m->psg, hsg + (size_t)b0 * 6, (size_t)nb * 6 * sizeof(float),
                              cudaMemcpyHostToDevice, st),
              "start/goal upload");
        MCUDA(cudaEventRecord(m->pin_ev, st), "proposal event");  // covers every copy out of `pin` so far
        voxelize_kernel<<<dim3(blocks_for((long long)m->G * m->G, kVoxRows), nb), kVoxRows, 0, st>>>(m->envs + b0, m->G,
                                                                                               m->pvox);
        MCUDA(cudaGetLastError(), "voxelize kernel");
        gmt_status s = forward(m, nb, m->pvox, m->psg, st);
        if (s != GMT_OK) return s;
        proposal_sample_kernel<<<nb, 1024, smem, st>>>(m->logits, m->Nc, m->C, m->penv + b0, count,
                                                                       65536, pitch, m->err);
        MCUDA(cudaGetLastError(), "proposal kernel");
    }
    int h = 0;
    MCUDA(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, st), "flag readback");
    MCUDA(cudaStreamSynchronize(st), "proposal");
    if (h) {
        cudaMemset(m->err, 0, sizeof(int));
        return mfail(GMT_ERR_INVALID, "a proposal sample exhausted its attempts (or a GEMM wait ran out)");
    }
    return GMT_OK;
}

}  // namespace

extern "C" {


gmt_status gmt_model_create(const gmt_model_config* cfg, gmt_model** out) {
    if (!cfg || !out) return mfail(GMT_ERR_INVALID, "config and out must be non-NULL");
    if (cfg->grid < 8 || cfg->grid > 64 || cfg->hidden < 64 || cfg->hidden % 64 || cfg->cells < 2 || cfg->cells > 32 ||
        cfg->max_batch < 1 || cfg->max_batch > 4096)
        return mfail(GMT_ERR_INVALID, "model config out of range");
    gmt_model* m = new gmt_model();
    m->G = cfg->grid; m->H = cfg->hidden; m->C = cfg->cells; m->maxB = cfg->max_batch; m->seed = cfg->seed;
    m->Din = m->G * m->G * m->G;
    m->Dz = m->H + 16;
    m->Nc = m->C * m->C * m->C;
    const int B = m->maxB;
    auto fail_delete = [&](gmt_status s) { delete m; return s; };
#define MK(p, n) do { cudaError_t e_ = mk(m, &m->p, (n)); if (e_ != cudaSuccess) return fail_delete(mcuda(e_, "model allocation")); } while (0)
    MK(W1, m->n(0)); MK(b1, m->n(1)); MK(W2, m->n(2)); MK(b2, m->n(3)); MK(W3, m->n(4)); MK(b3, m->n(5));
    MK(gW1, m->n(0)); MK(gb1, m->n(1)); MK(gW2, m->n(2)); MK(gb2, m->n(3)); MK(gW3, m->n(4)); MK(gb3, m->n(5));
    for (int i = 0; i < 6; ++i) {
        cudaError_t e = mk(m, &m->mom[i], m->n(i));
        if (e == cudaSuccess) e = mk(m, &m->vel[i], m->n(i));
        if (e != cudaSuccess) return fail_delete(mcuda(e, "model allocation"));
    }
    MK(W1b, m->n(0)); MK(W2b, m->n(2)); MK(W2tb, m->n(2)); MK(W3b, m->n(4)); MK(W3tb, m->n(4));
    MK(Xt, (size_t)B * m->Din); MK(H1, (size_t)B * m->H); MK(H1t, (size_t)B * m->H); MK(H2, (size_t)B * m->H);
    MK(Z, (size_t)B * m->Dz); MK(Zt, (size_t)B * m->Dz); MK(dlog, (size_t)B * m->Nc); MK(dlogt, (size_t)B * m->Nc);
    MK(dH2, (size_t)B * m->H); MK(dH2t, (size_t)B * m->H); MK(dH1p, (size_t)B * m->H); MK(dH1pt, (size_t)B * m->H);
    MK(logits, (size_t)B * m->Nc); MK(dZ, (size_t)B * m->Dz); MK(dH1, (size_t)B * m->H); MK(loss, B);
    m->ws_floats = (size_t)16 * std::max((size_t)B * m->H, (size_t)B * m->Dz) + (size_t)4 * B * m->Nc;
    MK(ws, m->ws_floats);
    MK(err, 1);
    MK(pvox, (size_t)B * m->Din);
    MK(psg, (size_t)B * 6);
#undef MK
    cudaStream_t st = 0;
    const uint32_t k0 = (uint32_t)(m->seed & 0xffffffffu), k1 = (uint32_t)(m->seed >> 32);
    const float stds[3] = {sqrtf(2.0f / (float)m->Din), sqrtf(2.0f / (float)m->H), sqrtf(1.0f / (float)m->Dz)};
    float* W[3] = {m->W1, m->W2, m->W3};
    for (int i = 0; i < 3; ++i) {
        init_normal_kernel<<<blocks_for(m->n(2 * i), 256), 256, 0, st>>>(W[i], m->n(2 * i), stds[i], k0, k1, i);
        cudaMemsetAsync(m->param(2 * i + 1), 0, m->n(2 * i + 1) * sizeof(float), st);
    }
    for (int i = 0; i < 6; ++i) {
        cudaMemsetAsync(m->mom[i], 0, m->n(i) * sizeof(float), st);
        cudaMemsetAsync(m->vel[i], 0, m->n(i) * sizeof(float), st);
    }
    cudaMemsetAsync(m->err, 0, sizeof(int), st);
    cudaError_t e = refresh_copies(m, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_delete(mcuda(e, "model initialisation"));
    *out = m;
    return GMT_OK;
}

void gmt_model_free(gmt_model* m) { delete m; }

gmt_status gmt_model_get_view(const gmt_model* m, gmt_model_view* v) {
    if (!m || !v) return mfail(GMT_ERR_INVALID, "model and view must be non-NULL");
    v->grid = m->G; v->hidden = m->H; v->cells = m->C; v->in_features = m->Din; v->z_features = m->Dz;
    v->n_cells = m->Nc; v->max_batch = m->maxB; v->step = m->step;
    v->W1 = m->W1; v->b1 = m->b1; v->W2 = m->W2; v->b2 = m->b2; v->W3 = m->W3; v->b3 = m->b3;
    v->gW1 = m->gW1; v->gb1 = m->gb1; v->gW2 = m->gW2; v->gb2 = m->gb2; v->gW3 = m->gW3; v->gb3 = m->gb3;
    v->W1_bf16 = m->W1b; v->W2_bf16 = m->W2b; v->W3_bf16 = m->W3b;
    v->logits = m->logits; v->loss = m->loss;
    v->H1 = m->H1; v->H2 = m->H2; v->Z = m->Z; v->dlog = m->dlog; v->dH2 = m->dH2; v->dH1 = m->dH1p;
    return GMT_OK;
}

gmt_status gmt_voxelize(int32_t B, const gmt_boxes* boxes, int32_t grid, void* voxels, gmt_stream stream) {
    if (B < 1 || !boxes || !voxels || grid < 1 || grid > 64) return mfail(GMT_ERR_INVALID, "bad voxelize arguments");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<EnvBoxes> h(B);
    for (int b = 0; b < B; ++b) {
        if (boxes[b].count < 0 || (boxes[b].count > 0 && (!boxes[b].lo || !boxes[b].hi)))
            return mfail(GMT_ERR_INVALID, "bad box arrays");
        h[b] = EnvBoxes{boxes[b].count, boxes[b].lo, boxes[b].hi};
    }
    EnvBoxes* d = nullptr;
    MCUDA(cudaMallocAsync((void**)&d, B * sizeof(EnvBoxes), st), "voxelize descriptors");
    MCUDA(cudaMemcpyAsync(d, h.data(), B * sizeof(EnvBoxes), cudaMemcpyHostToDevice, st), "voxelize descriptors");
    voxelize_kernel<<<dim3(blocks_for((long long)grid * grid, kVoxRows), B), kVoxRows, 0, st>>>(d, grid, (bf16*)voxels);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(d, st);
    MCUDA(e, "voxelize kernel");
    MCUDA(cudaStreamSynchronize(st), "voxelize");
    return GMT_OK;
}

gmt_status gmt_model_forward(gmt_model* m, int32_t B, const void* voxels, const float* start_goal, float* logits,
                             gmt_stream stream) {
    if (!m || B < 1 || B > m->maxB || !voxels || !start_goal) return mfail(GMT_ERR_INVALID, "bad forward arguments");
    cudaStream_t st = (cudaStream_t)stream;
    gmt_status s = forward(m, B, (const bf16*)voxels, start_goal, st);
    if (s != GMT_OK) return s;
    if (logits)
        MCUDA(cudaMemcpyAsync(logits, m->logits, (size_t)B * m->Nc * sizeof(float), cudaMemcpyDeviceToDevice, st),
              "logits copy");
    return check_err(m, st);
}

gmt_status gmt_model_backward(gmt_model* m, int32_t B, const void* voxels, const float* start_goal,
                              const float* target, float* mean_loss, gmt_stream stream) {
    if (!m || B < 1 || B > m->maxB || !voxels || !start_goal || !target)
        return mfail(GMT_ERR_INVALID, "bad backward arguments");
    cudaStream_t st = (cudaStream_t)stream;
    gmt_status s = forward(m, B, (const bf16*)voxels, start_goal, st);
    if (s == GMT_OK) s = backward(m, B, (const bf16*)voxels, target, st);
    if (s != GMT_OK) return s;
    std::vector<float> l(B);
    MCUDA(cudaMemcpyAsync(l.data(), m->loss, B * sizeof(float), cudaMemcpyDeviceToHost, st), "loss readback");
    s = check_err(m, st);
    if (s != GMT_OK) return s;
    if (mean_loss) {
        double a = 0.0;
        for (float x : l) a += x;
        *mean_loss = (float)(a / B);
    }
    return GMT_OK;
}

gmt_status gmt_model_train_step(gmt_model* m, int32_t B, const void* voxels, const float* start_goal,
                                const float* target, float lr, float weight_decay, float* mean_loss,
                                gmt_stream stream) {
    gmt_status s = gmt_model_backward(m, B, voxels, start_goal, target, mean_loss, stream);
    if (s != GMT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
    bf16* copies[6] = {m->W1b, nullptr, m->W2b, nullptr, m->W3b, nullptr};
    for (int i = 0; i < 6; ++i) {
        const float wd = (i % 2 == 0) ? weight_decay : 0.0f;
        adamw_kernel<<<blocks_for(m->n(i), 256), 256, 0, st>>>(m->param(i), m->grad(i), m->mom[i], m->vel[i], m->n(i),
                                                               lr, b1, b2, eps, wd, c1, c2, copies[i]);
    }
    MCUDA(cudaGetLastError(), "AdamW");
    MCUDA(transpose(m->W2b, m->H, m->H, m->W2tb, st), "transpose");
    MCUDA(transpose(m->W3b, m->Nc, m->Dz, m->W3tb, st), "transpose");
    MCUDA(cudaStreamSynchronize(st), "train step");
    return GMT_OK;
}

gmt_status gmt_model_save(const gmt_model* m, const char* path) {
    if (!m || !path) return mfail(GMT_ERR_INVALID, "model and path must be non-NULL");
    FILE* f = fopen(path, "wb");
    if (!f) return mfail(GMT_ERR_INVALID, std::string("cannot open ") + path);
    const int32_t hdr[6] = {0x474d5450 /*'GMTP'*/, m->G, m->H, m->C, m->maxB, 1};
    fwrite(hdr, sizeof(hdr), 1, f);
    fwrite(&m->step, sizeof(m->step), 1, f);
    fwrite(&m->seed, sizeof(m->seed), 1, f);
    std::vector<float> buf;
    for (int i = 0; i < 6; ++i) {
        float* srcs[3] = {const_cast<gmt_model*>(m)->param(i), m->mom[i], m->vel[i]};
        for (float* src : srcs) {
            buf.resize(m->n(i));
            if (cudaMemcpy(buf.data(), src, m->n(i) * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
                fclose(f);
                return mfail(GMT_ERR_CUDA, "checkpoint copy");
            }
            fwrite(buf.data(), sizeof(float), buf.size(), f);
        }
    }
    fclose(f);
    return GMT_OK;
}

gmt_status gmt_model_load(gmt_model* m, const char* path) {
    if (!m || !path) return mfail(GMT_ERR_INVALID, "model and path must be non-NULL");
    FILE* f = fopen(path, "rb");
    if (!f) return mfail(GMT_ERR_INVALID, std::string("cannot open ") + path);
    int32_t hdr[6];
    if (fread(hdr, sizeof(hdr), 1, f) != 1 || hdr[0] != 0x474d5450 || hdr[1] != m->G || hdr[2] != m->H ||
        hdr[3] != m->C) {
        fclose(f);
        return mfail(GMT_ERR_INVALID, "checkpoint does not match the model shape");
    }
    if (fread(&m->step, sizeof(m->step), 1, f) != 1 || fread(&m->seed, sizeof(m->seed), 1, f) != 1) {
        fclose(f);
        return mfail(GMT_ERR_INVALID, "truncated checkpoint");
    }
    std::vector<float> buf;
    for (int i = 0; i < 6; ++i) {
        float* dsts[3] = {m->param(i), m->mom[i], m->vel[i]};
        for (float* dst : dsts) {
            buf.resize(m->n(i));
            if (fread(buf.data(), sizeof(float), buf.size(), f) != buf.size()) {
                fclose(f);
                return mfail(GMT_ERR_INVALID, "truncated checkpoint");
            }
            if (cudaMemcpy(dst, buf.data(), m->n(i) * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
                fclose(f);
                return mfail(GMT_ERR_CUDA, "checkpoint copy");
            }
        }
    }
    fclose(f);
    cudaError_t e = refresh_copies(m, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return mcuda(e, "checkpoint refresh");
    return GMT_OK;
}

gmt_status gmt_path_histogram(const float* X, int32_t pitch, const int32_t* path, int32_t len, int32_t cells,
                              float spacing, float eps, float* hist, gmt_stream stream) {
    if (!X || !path || !hist || len < 0 || cells < 1 || !(spacing > 0.0f))
        return mfail(GMT_ERR_INVALID, "bad histogram arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = cells * cells * cells;
    const size_t smem = (size_t)n * sizeof(float);
    if (smem > 200 * 1024) return mfail(GMT_ERR_INVALID, "cells^3 too large for the histogram kernel");
    static std::atomic<bool> attr_set{false};
    if (!attr_set.load(std::memory_order_relaxed)) {
        MCUDA(cudaFuncSetAttribute(path_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
              "histogram kernel attribute");
        attr_set.store(true, std::memory_order_relaxed);
    }
    path_hist_kernel<<<1, 256, smem, st>>>(X, pitch, path, len, cells, spacing, eps, hist);
    MCUDA(cudaGetLastError(), "histogram kernel");
    return GMT_OK;
}

gmt_status gmt_propose(gmt_model* m, const gmt_space* space, const gmt_boxes* boxes, const float* start,
                       const float* goal, int32_t count, uint64_t seed, float* samples, int32_t pitch,
                       gmt_stream stream) {
    if (!space || !start || !goal) return mfail(GMT_ERR_INVALID, "bad proposal arguments");
    float sg[6];
    for (int a = 0; a < 3; ++a) { sg[a] = start[a]; sg[3 + a] = goal[a]; }
    return propose_impl(m, 1, space, boxes, sg, count, &seed, samples, pitch, stream);
}

gmt_status gmt_propose_batch(gmt_model* m, int32_t B, const gmt_space* spaces, const gmt_boxes* boxes,
                             const float* start_goal, int32_t count, const uint64_t* seeds, float* samples,
                             int32_t pitch, gmt_stream stream) {
    return propose_impl(m, B, spaces, boxes, start_goal, count, seeds, samples, pitch, stream);
}

}  // extern "C"
