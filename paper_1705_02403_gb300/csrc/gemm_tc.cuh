// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05) for
// sm_103a, written with inline PTX:
//   C[M, N] = A[M, K] . B[N, K]^T   (both operands K-major, row-major in memory)
//
// One CTA of 128 threads computes a 128 x 128 tile of C (optionally a K-slice
// of it, for split-K):
//   - warp 0 allocates 128 TMEM columns (the FP32 accumulator: 128 lanes x 128
//     columns) and frees them at the end;
//   - one thread of warp 0 is the TMA producer: 64-wide K-blocks of A and B are
//     loaded with cp.async.bulk.tensor into a ring of STAGES shared-memory
//     buffers in the 128-byte-swizzled K-major layout the MMA reads (6 for
//     deep K; 3 for short K, so that two CTAs share an SM and one's epilogue
//     overlaps the other's loads);
//   - one thread of warp 1 issues tcgen05.mma (kind::f16, M = 128, N = 128,
//     K = 16 per instruction, 4 per K-block) and returns each stage to the
//     producer with tcgen05.commit on the stage's "empty" mbarrier;
//   - after the last commit, all four warps read their 32 accumulator lanes
//     with tcgen05.ld (32 columns at a time) into the ring's shared memory,
//     which the MMAs no longer read, and each warp then writes its 32 rows
//     128 bytes at a time (one row segment per warp store) with the epilogue.
// Every mbarrier wait is bounded: a wait that runs out sets an error flag and
// the CTA stops issuing work, waits (bounded) for copies it issued, releases
// its TMEM and returns.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gmtk {

constexpr int kGemmBM = 128, kGemmBN = 128, kGemmBK = 64;
constexpr int kGemmStagesDeep = 6, kGemmStagesShort = 3;
// Epilogue staging: each row of the FP32 tile padded to 129 floats, so the 32
// lanes of a warp (32 rows) write one column in 32 different banks.
constexpr int kGemmStagePitch = kGemmBN + 1;
constexpr int kGemmTileBytes = kGemmBM * kGemmBK * 2;  // 16 KB per operand tile
__host__ __device__ constexpr int gemm_smem_bytes(int stages) {
    return 2 * stages * kGemmTileBytes + 1024 /*align*/ + 256 /*barriers*/;
}
static_assert(kGemmBM * kGemmStagePitch * 4 <= 2 * kGemmStagesShort * kGemmTileBytes,
              "the epilogue staging fits the operand ring");
constexpr long long kGemmSpinLimit = 1ll << 26;

enum GemmEpilogue { kEpiStoreF32 = 0, kEpiBiasReluBF16 = 1, kEpiBiasF32 = 2, kEpiPartialF32 = 3 };

struct GemmArgs {
    int M, N, K;
    int k_blocks_per_split;  // K-blocks (of 64) handled by one CTA along gridDim.z
    int epilogue;
    float* C;                // FP32 output [M, ldc] (or partials [splits][M][ldc])
    __nv_bfloat16* Cb;       // BF16 output [M, ldc] (kEpiBiasReluBF16)
    const float* bias;       // [N] or NULL
    int ldc;
    int* error;              // set to 1 when a bounded wait runs out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One poll of the barrier's phase with the given parity.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false if it ran out (and the error flag was set).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* error) {
    for (long long i = 0; i < kGemmSpinLimit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if ((i & 1023) == 1023 && *(volatile int*)error) return false;
    }
    atomicExch(error, 1);
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzled
// layout (rows of 128 bytes, 8-row groups 1024 bytes apart): start address,
// leading byte offset 16 (unused by this layout), stride byte offset 1024,
// descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5
// = 1), BF16 A and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t mma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int STAGES>
__global__ void __launch_bounds__(128, 1) gemm_tn_bf16_kernel(const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmB, GemmArgs g) {
    constexpr int kGemmStages = STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;
    uint8_t* sB = base + kGemmStages * kGemmTileBytes;
    uint64_t* full = (uint64_t*)(base + 2 * kGemmStages * kGemmTileBytes);
    uint64_t* empty = full + kGemmStages;
    uint64_t* done = empty + kGemmStages;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kGemmBM, n0 = blockIdx.y * kGemmBN;
    const int kb_total = (g.K + kGemmBK - 1) / kGemmBK;
    const int kb0 = blockIdx.z * g.k_blocks_per_split;
    const int kb1 = min(kb_total, kb0 + g.k_blocks_per_split);
    const int nkb = max(0, kb1 - kb0);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kGemmStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        // TMA producer
        int issued = 0;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % kGemmStages, round = i / kGemmStages;
            if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1, g.error)) break;
            mbar_expect_tx(&full[s], 2 * kGemmTileBytes);
            const int kx = (kb0 + i) * kGemmBK;
            tma_load_2d(sA + s * kGemmTileBytes, &tmA, kx, m0, &full[s]);
            tma_load_2d(sB + s * kGemmTileBytes, &tmB, kx, n0, &full[s]);
            ++issued;
        }
        if (issued < nkb) {
            // stopped early: let the copies already issued land before leaving
            for (int i = max(0, issued - kGemmStages); i < issued; ++i)
                mbar_wait(&full[i % kGemmStages], (i / kGemmStages) & 1, g.error);
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        const uint32_t idesc = mma_idesc_bf16(kGemmBM, kGemmBN);
        bool ok = true;
        for (int i = 0; i < nkb && ok; ++i) {
            const int s = i % kGemmStages, round = i / kGemmStages;
            if (!mbar_wait(&full[s], round & 1, g.error)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA + s * kGemmTileBytes), b0 = smem_u32(sB + s * kGemmTileBytes);
#pragma unroll
            for (int kk = 0; kk < kGemmBK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        mma_commit(done);
    }
    __syncwarp();
    // epilogue: every warp waits for the accumulator, then reads its 32 lanes;
    // the decision is made warp-uniform because tcgen05.ld is warp-collective
    const bool waited = nkb > 0 && mbar_wait(done, 0, g.error);
    const bool have = __all_sync(0xffffffffu, waited && *(volatile int*)g.error == 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (have) {
        // the warp's 32 accumulator rows into shared memory (row-major, padded) ...
        float* stage = reinterpret_cast<float*>(base) + warp * 32 * kGemmStagePitch;
        for (int c = 0; c < kGemmBN; c += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) stage[lane * kGemmStagePitch + c + j] = v[j];
        }
        __syncwarp();
        // ... then out, one 32-column row segment per warp store
        const float* biasp = g.bias;
        for (int r = 0; r < 32; ++r) {
            const int row = m0 + warp * 32 + r;
            if (row >= g.M) break;
            for (int c = 0; c < kGemmBN; c += 32) {
                const int col = n0 + c + lane;
                if (col >= g.N) continue;
                const float x = stage[r * kGemmStagePitch + c + lane];
                if (g.epilogue == kEpiPartialF32) {
                    g.C[(size_t)blockIdx.z * g.M * g.ldc + (size_t)row * g.ldc + col] = x;
                } else if (g.epilogue == kEpiBiasReluBF16) {
                    g.Cb[(size_t)row * g.ldc + col] = __float2bfloat16_rn(fmaxf(x + (biasp ? biasp[col] : 0.0f), 0.0f));
                } else {
                    g.C[(size_t)row * g.ldc + col] = x + ((g.epilogue == kEpiBiasF32 && biasp) ? biasp[col] : 0.0f);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

}  // namespace gmtk
