// tcgen05 GEMM of the surrogate: C[M x N] = A[M x K] * B[N x K]^T, BF16
// operands, FP32 accumulation in tensor memory, fused epilogue.
//
// One CTA of 8 warps computes a 128 x NT tile (NT = 128 or 256):
//   * TMA (cp.async.bulk.tensor.2d, 128-byte swizzle) brings 64-wide K chunks
//     of A (128 x 64) and B (NT x 64) into a ring of kStages shared-memory
//     stages; an mbarrier per stage counts the arriving bytes.
//   * One thread issues tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = NT,
//     K = 16 per instruction, four per chunk) into an FP32 accumulator of NT
//     tensor-memory columns, and tcgen05.commit releases each stage back to
//     the loader once the tensor cores have read it.
//   * After the last chunk the eight warps read the accumulator with
//     tcgen05.ld.32x32b (warp w: lanes 32*(w%4).., column half w/4) and apply
//     the epilogue through a shared-memory transpose (coalesced stores).
// Every mbarrier wait is bounded: on timeout the kernel records an error in
// g_tc_error, stops issuing work, waits (bounded) for its TMA loads in flight
// and for the tensor cores, frees its tensor memory and returns.  The poll
// limit of the main loop's waits is g_tc_wait_limit (settable, so that a
// test can make a wait run out); the draining waits keep the fixed kSpin.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace chert {
namespace gemm {

__device__ int g_tc_error;          // 0 = ok; 1 = a main-loop wait timed out, 2 = the accumulator wait,
                                    // 3 = a TMA load still in flight after the drain

namespace tc {

constexpr int kStages = 3;
constexpr int kKChunk = 64;          // bf16 elements = 128 bytes = one swizzle row
constexpr long long kSpin = 1 << 22; // bounded waits
}  // namespace tc

__device__ long long g_tc_wait_limit = tc::kSpin;   // polls of the main loop's waits

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait on an mbarrier phase (at most `limit` polls); returns false on
// timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kSpin) {
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzle
// layout TMA writes: rows 128 bytes apart, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;                  // start address
    d |= (uint64_t(16 >> 4) & 0x3FFFull) << 16;    // leading byte offset (unused when swizzled)
    d |= (uint64_t(1024 >> 4) & 0x3FFFull) << 32;  // stride byte offset: 8 rows x 128 B
    d |= 1ull << 46;                               // descriptor version
    d |= 2ull << 61;                               // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = nt.
__host__ __device__ constexpr uint32_t instr_desc(int nt) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(nt >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

template <int NT>
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(slot)), "n"(NT));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

template <int NT>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NT));
}

__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 32 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int NT>
struct Smem {
    alignas(1024) __nv_bfloat16 a[kStages][128 * kKChunk];
    alignas(1024) __nv_bfloat16 b[kStages][NT * kKChunk];
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t done;
    uint32_t tmem;
};

template <int NT>
__global__ void __launch_bounds__(256, 1) nt_tc_kernel(const __grid_constant__ CUtensorMap ta,
                                                       const __grid_constant__ CUtensorMap tb, int M, int N,
                                                       int K, Epilogue e) {
    extern __shared__ __align__(1024) unsigned char raw[];
    Smem<NT>& s = *reinterpret_cast<Smem<NT>*>(
        (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * NT;
    const int nk = (K + kKChunk - 1) / kKChunk;
    if (warp == 0) tmem_alloc<NT>(&s.tmem);
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) { mbar_init(&s.full[i], 1); mbar_init(&s.empty[i], 1); }
        mbar_init(&s.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s.tmem;
    constexpr uint32_t kBytes = (128 + NT) * kKChunk * 2;
    __shared__ int s_fail;
    if (tid == 0) {
        s_fail = 0;
        const uint32_t idesc = instr_desc(NT);
        const long long limit = g_tc_wait_limit;
        bool ok = true;
        // pending[st]: the K chunk whose TMA load into stage st has not been
        // waited for yet, or -1
        int pending[kStages];
        for (int i = 0; i < kStages; ++i) pending[i] = -1;
        const int pre = nk < kStages ? nk : kStages;
        for (int c = 0; c < pre; ++c) {
            mbar_expect_tx(&s.full[c], kBytes);
            tma_load_2d(s.a[c], &ta, c * kKChunk, m0, &s.full[c]);
            tma_load_2d(s.b[c], &tb, c * kKChunk, n0, &s.full[c]);
            pending[c] = c;
        }
        int issued = 0;
        for (int c = 0; c < nk && ok; ++c) {
            const int st = c % kStages;
            ok = mbar_wait(&s.full[st], (c / kStages) & 1, limit);
            if (!ok) break;
            pending[st] = -1;
            ++issued;
            fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kKChunk / 16; ++kk)
                mma_bf16(tmem, smem_desc(s.a[st] + kk * 16), smem_desc(s.b[st] + kk * 16), idesc,
                         (c > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&s.empty[st]);
            const int nxt = c + kStages;
            if (nxt < nk) {
                ok = mbar_wait(&s.empty[st], (c / kStages) & 1, limit);   // tensor cores done with this stage
                if (!ok) break;
                mbar_expect_tx(&s.full[st], kBytes);
                tma_load_2d(s.a[st], &ta, nxt * kKChunk, m0, &s.full[st]);
                tma_load_2d(s.b[st], &tb, nxt * kKChunk, n0, &s.full[st]);
                pending[st] = nxt;
            }
        }
        int code = ok ? 0 : 1;
        if (!ok) {
            // the loads in flight land before the CTA gives up its shared memory
            for (int i = 0; i < kStages; ++i)
                if (pending[i] >= 0 && !mbar_wait(&s.full[i], (pending[i] / kStages) & 1)) code = 3;
        }
        if (issued)
            mma_commit(&s.done);            // arrives once the issued MMAs are complete
        else
            mbar_arrive(&s.done);           // nothing in the tensor cores
        if (code) { s_fail = 1; atomicExch(&g_tc_error, code); }
    }
    // all threads: wait for the accumulator (bounded; commits arrive even after a failure)
    const bool done = mbar_wait(&s.done, 0);
    __syncthreads();
    if (!done && tid == 0) atomicExch(&g_tc_error, 2);
    fence_after_sync();
    if (done && !s_fail) {
        // Eight warps: warp w reads accumulator lanes 32*(w%4).. (its rows) and
        // the column half w/4.  A 32 x 32 block is read from tensor memory
        // (one row per thread), transposed through a padded shared-memory tile
        // (the operand stages are free once the MMAs are done), and the
        // epilogue runs with the lanes along the row, so every global access
        // is a coalesced row segment.
        const int quarter = warp & 3, half = warp >> 2;
        float* stg = reinterpret_cast<float*>(s.a[0]) + warp * 32 * 33;
        const uint32_t lane_base = tmem + (uint32_t(quarter * 32) << 16);
        const int row0 = m0 + quarter * 32;
        for (int c0 = half * (NT / 2); c0 < (half + 1) * (NT / 2); c0 += 32) {
            float v[32];
            tmem_ld32(lane_base + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) stg[lane * 33 + i] = v[i];
            __syncwarp();
            for (int r = 0; r < 32; ++r)
                if (row0 + r < M) epilogue_store(e, M, N, row0 + r, n0 + c0 + lane, stg[r * 33 + lane]);
            __syncwarp();
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc<NT>(tmem);
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeFn encoder(const char** why) {
    static EncodeFn fn = nullptr;
    static char msg[160] = "";
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        const cudaError_t e =
            cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && p) fn = reinterpret_cast<EncodeFn>(p);
        else snprintf(msg, sizeof(msg), "cuTensorMapEncodeTiled not available (%s, query %d)",
                      cudaGetErrorString(e), (int)q);
    }
    if (why) *why = msg;
    return fn;
}

// 2D map over a row-major bf16 matrix [rows x cols] with row pitch ld; boxes
// of 64 columns x box_rows rows, 128-byte swizzle, zero fill outside.
inline int make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int cols, int ld, int box_rows) {
    const char* why = nullptr;
    EncodeFn fn = encoder(&why);
    if (!fn) {
        set_error("surrogate GEMM: %s", why);
        return CHERT_ECUDA;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKChunk, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("surrogate GEMM: cuTensorMapEncodeTiled failed (%d) for %d x %d, ld %d", (int)r, rows, cols, ld);
        return CHERT_ECUDA;
    }
    return CHERT_OK;
}

inline bool& tensor_cores_enabled() {
    static bool on = true;
    return on;
}

// Reads and clears the error flag of the tensor-core kernel (synchronises s).
inline int check_and_clear(cudaStream_t s, const char* who) {
    int h = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&h, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (h) {
        const int z = 0;
        cudaMemcpyToSymbolAsync(g_tc_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
        set_error("%s: a tensor-core GEMM gave up waiting (code %d)", who, h);
        return CHERT_ETIMEOUT;
    }
    return CHERT_OK;
}

// Launch if the shapes suit the tensor-core kernel; returns 1 when launched,
// 0 when the caller should use the CUDA-core kernel, or a negative status.
inline int try_nt(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                  const Epilogue& e, cudaStream_t s) {
    if (!tensor_cores_enabled()) return 0;
    if (M < 128 || K < 16 || (N % 128) != 0) return 0;
    if ((lda % 8) || (ldb % 8) || (reinterpret_cast<uintptr_t>(A) % 16) || (reinterpret_cast<uintptr_t>(B) % 16))
        return 0;
    const int nt = (N % 256 == 0 && (long long)((M + 127) / 128) * (N / 256) >= 148) ? 256 : 128;
    CUtensorMap ta, tb;
    int rc = make_map(&ta, A, M, K, lda, 128);
    if (!rc) rc = make_map(&tb, B, N, K, ldb, nt);
    if (rc) return rc;
    const dim3 grid(N / nt, (M + 127) / 128);
    if (grid.y > 65535u) {
        set_error("surrogate GEMM: M=%d exceeds one launch; split the batch", M);
        return CHERT_EINVAL;
    }
    if (nt == 256) {
        const size_t smem = sizeof(Smem<256>) + 1024;
        cudaError_t err = cudaFuncSetAttribute(nt_tc_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return cuda_fail(err, "surrogate GEMM (tcgen05)");
        nt_tc_kernel<256><<<grid, 256, smem, s>>>(ta, tb, M, N, K, e);
    } else {
        const size_t smem = sizeof(Smem<128>) + 1024;
        cudaError_t err = cudaFuncSetAttribute(nt_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return cuda_fail(err, "surrogate GEMM (tcgen05)");
        nt_tc_kernel<128><<<grid, 256, smem, s>>>(ta, tb, M, N, K, e);
    }
    rc = launch_check("surrogate GEMM (tcgen05)");
    return rc ? rc : 1;
}

}  // namespace tc
}  // namespace gemm
}  // namespace chert
