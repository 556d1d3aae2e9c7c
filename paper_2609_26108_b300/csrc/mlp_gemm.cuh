// GEMM C[M x N] = A[M x K] * B[N x K]^T of the surrogate (BF16 operands, FP32
// accumulation) with the fused epilogues the MLP needs.  The tcgen05 kernel
// (mlp_tc.cuh) takes the large shapes; the plain CUDA-core kernel here
// (shared-memory tiles of 64 x 64 outputs, 4 x 4 per thread) takes the rest.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace chert {
namespace gemm {

enum Mode { kPlain = 0, kBias = 1, kBiasSilu = 2, kDsilu = 3 };

struct Epilogue {
    int mode;
    const float* bias;       // [N]                      (kBias, kBiasSilu)
    float* z_out;            // [M x N] pre-activation   (kBiasSilu, optional)
    __nv_bfloat16* h_out;    // [M x N] bf16 result      (kBiasSilu, kDsilu)
    float* y_out;            // [M x N] fp32 result      (kPlain, kBias)
    const float* z_in;       // [M x N] pre-activation   (kDsilu)
    float* g_out;            // [M x N] fp32 result      (kDsilu)
};

// SiLU and its derivative with the fast exponential and division intrinsics
// (their relative error, ~1e-6, is far below the bfloat16 rounding that follows).
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = __fdividef(1.0f, 1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ void epilogue_store(const Epilogue& e, int M, int N, int m, int n, float c) {
    if (m >= M || n >= N) return;
    const size_t i = (size_t)m * N + n;
    switch (e.mode) {
        case kPlain: e.y_out[i] = c; break;
        case kBias: e.y_out[i] = c + e.bias[n]; break;
        case kBiasSilu: {
            const float z = c + e.bias[n];
            if (e.z_out) e.z_out[i] = z;
            e.h_out[i] = __float2bfloat16_rn(silu_f(z));
            break;
        }
        default: {
            const float g = c * dsilu_f(e.z_in[i]);
            e.g_out[i] = g;
            e.h_out[i] = __float2bfloat16_rn(g);
        }
    }
}

__global__ void __launch_bounds__(256) nt_simt_kernel(const __nv_bfloat16* __restrict__ A, int lda,
                                                      const __nv_bfloat16* __restrict__ B, int ldb,
                                                      int M, int N, int K, Epilogue e) {
    __shared__ float As[16][65], Bs[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            const int kk = t & 15, r = t >> 4;
            const int m = m0 + r, n = n0 + r, k = k0 + kk;
            As[kk][r] = (m < M && k < K) ? __bfloat162float(A[(size_t)m * lda + k]) : 0.0f;
            Bs[kk][r] = (n < N && k < K) ? __bfloat162float(B[(size_t)n * ldb + k]) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) epilogue_store(e, M, N, m0 + ty * 4 + i, n0 + tx * 4 + j, acc[i][j]);
}

}  // namespace gemm
}  // namespace chert

#include "mlp_tc.cuh"

namespace chert {
namespace gemm {

// tcgen05 kernel when the shapes allow it (M >= 128, N a multiple of 128,
// K >= 16, 16-byte aligned rows), the CUDA-core kernel otherwise.
inline int nt(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
              const Epilogue& e, cudaStream_t s, bool allow_tc = true) {
    if (M <= 0 || N <= 0 || K <= 0) return CHERT_OK;
    if (allow_tc) {
        const int r = tc::try_nt(A, lda, B, ldb, M, N, K, e, s);
        if (r != 0) return r < 0 ? r : CHERT_OK;
    }
    const dim3 grid((M + 63) / 64, (N + 63) / 64);
    if (grid.y > 65535u) {
        set_error("surrogate GEMM: N=%d too large for one launch", N);
        return CHERT_EINVAL;
    }
    nt_simt_kernel<<<grid, 256, 0, s>>>(A, lda, B, ldb, M, N, K, e);
    return launch_check("surrogate GEMM");
}

}  // namespace gemm
}  // namespace chert
