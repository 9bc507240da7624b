// Learned sampling proposal: the BF16 tensor-core GEMM launcher and the C ABI
// entry point that exposes it (gmt_gemm_bf16).  The network, its training and
// the proposal sampler build on these (proposal.cu).
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

#include "gemm_tc.cuh"
#include "internal.h"

namespace gmtk {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// Tensor map of a row-major BF16 matrix [rows, cols] (cols contiguous) read in
// boxes of 64 columns x 128 rows, 128-byte swizzle, zero fill out of range.
cudaError_t make_map(CUtensorMap* map, const void* ptr, int rows, int cols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if (((uintptr_t)ptr & 15) != 0 || (cols * 2) % 16 != 0) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kGemmBK, (cuuint32_t)kGemmBM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Sum of split-K partials [splits][M][N] plus the epilogue.
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, int M, int N, int epilogue,
                                     const float* __restrict__ bias, float* __restrict__ C,
                                     __nv_bfloat16* __restrict__ Cb, int ldc) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)M * N) return;
    const int row = (int)(t / N), col = (int)(t % N);
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * M * N + t];
    if (epilogue == kEpiBiasReluBF16) {
        const float x = fmaxf(s + (bias ? bias[col] : 0.0f), 0.0f);
        Cb[(size_t)row * ldc + col] = __float2bfloat16_rn(x);
    } else {
        C[(size_t)row * ldc + col] = s + ((epilogue == kEpiBiasF32 && bias) ? bias[col] : 0.0f);
    }
}

}  // namespace

// C = A . B^T with A [M, K], B [N, K] BF16 row-major; epilogue as GemmEpilogue.
// splits > 1 splits K across gridDim.z into `partial` ([splits][M][N] FP32)
// and reduces deterministically.
cudaError_t gemm_bf16_tn(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* B, int epilogue,
                         const float* bias, float* C, __nv_bfloat16* Cb, int ldc, int splits, float* partial,
                         int* error, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0 || K % 8 != 0) return cudaErrorInvalidValue;
    static std::atomic<bool> attr_set{false};  // setting it twice is harmless
    if (!attr_set.load(std::memory_order_relaxed)) {
        cudaError_t e = cudaFuncSetAttribute(gemm_tn_bf16_kernel<kGemmStagesDeep>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             gemm_smem_bytes(kGemmStagesDeep));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(gemm_tn_bf16_kernel<kGemmStagesShort>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_smem_bytes(kGemmStagesShort));
        if (e != cudaSuccess) return e;
        attr_set.store(true, std::memory_order_relaxed);
    }
    CUtensorMap ta, tb;
    cudaError_t e = make_map(&ta, A, M, K);
    if (e == cudaSuccess) e = make_map(&tb, B, N, K);
    if (e != cudaSuccess) return e;
    const int kb = (K + kGemmBK - 1) / kGemmBK;
    if (splits < 1) splits = 1;
    if (splits > kb) splits = kb;
    const int per = (kb + splits - 1) / splits;
    splits = (kb + per - 1) / per;  // every split gets at least one K-block
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = M; g.N = N; g.K = K; g.k_blocks_per_split = per; g.error = error; g.bias = bias; g.ldc = ldc;
    dim3 grid((M + kGemmBM - 1) / kGemmBM, (N + kGemmBN - 1) / kGemmBN, splits);
    // short K: a shallow ring, two CTAs per SM
    const bool shallow = per <= 2 * kGemmStagesShort;
    auto launch = [&](const GemmArgs& a) {
        if (shallow)
            gemm_tn_bf16_kernel<kGemmStagesShort><<<grid, 128, gemm_smem_bytes(kGemmStagesShort), st>>>(ta, tb, a);
        else
            gemm_tn_bf16_kernel<kGemmStagesDeep><<<grid, 128, gemm_smem_bytes(kGemmStagesDeep), st>>>(ta, tb, a);
    };
    if (splits == 1) {
        g.epilogue = epilogue; g.C = C; g.Cb = Cb;
        launch(g);
        return cudaGetLastError();
    }
    if (!partial) return cudaErrorInvalidValue;
    g.epilogue = kEpiPartialF32; g.C = partial; g.ldc = N;
    launch(g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long total = (long long)M * N;
    splitk_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(partial, splits, M, N, epilogue, bias, C, Cb,
                                                                          ldc);
    return cudaGetLastError();
}

}  // namespace gmtk

extern "C" gmt_status gmt_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, const void* B, int32_t epilogue,
                                    const float* bias, float* C, void* C_bf16, int32_t splits, float* workspace,
                                    int32_t* error_flag, gmt_stream stream) {
    if (M <= 0 || N <= 0 || K <= 0 || K % 8 != 0 || !A || !B || !error_flag) {
        gmtk::record_error("gmt_gemm_bf16: need M, N, K > 0, K % 8 == 0, non-NULL A, B, error_flag");
        return GMT_ERR_INVALID;
    }
    if (epilogue < 0 || epilogue > 2 || (epilogue == 1 ? !C_bf16 : !C)) {
        gmtk::record_error("gmt_gemm_bf16: bad epilogue or missing output");
        return GMT_ERR_INVALID;
    }
    if (splits > 1 && !workspace) {
        gmtk::record_error("gmt_gemm_bf16: split-K needs a workspace of splits*M*N floats");
        return GMT_ERR_INVALID;
    }
    cudaError_t e = gmtk::gemm_bf16_tn(M, N, K, (const __nv_bfloat16*)A, (const __nv_bfloat16*)B, epilogue, bias, C,
                                       (__nv_bfloat16*)C_bf16, N, splits, workspace, error_flag, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        gmtk::record_error((std::string("gmt_gemm_bf16: ") + cudaGetErrorString(e)).c_str());
        return GMT_ERR_CUDA;
    }
    return GMT_OK;
}
