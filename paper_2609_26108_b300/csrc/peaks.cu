// Measured arithmetic peaks of this GPU for the rooflines of the cache build
// (FP32 for the scan, FP64 for the double-precision build): a grid of several
// CTAs per SM, each thread running eight independent multiply-add chains, so
// that neither latency nor occupancy limits the rate.  Timed with events on
// the caller's stream.
#include <math.h>

#include "common.cuh"

namespace chert {
namespace {

__device__ float g_sink_f;
__device__ double g_sink_d;
__device__ __forceinline__ void sink(float v) { g_sink_f = v; }
__device__ __forceinline__ void sink(double v) { g_sink_d = v; }

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(int iters, T a, T b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = T(t + k) * T(1e-7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == T(-1)) sink(s);           // never true for these inputs; keeps the chains live
}

}  // namespace
}  // namespace chert

extern "C" int chert_fma_rate(int precision, int iters, double* flops_per_s, void* stream) {
    using namespace chert;
    CHERT_REQUIRE(flops_per_s && iters >= 1, "chert_fma_rate: bad arguments");
    CHERT_REQUIRE(precision == CHERT_FP64 || precision == CHERT_FP32, "chert_fma_rate: precision=%d", precision);
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "chert_fma_rate: device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = n_sm * 8, threads = 256;
    cudaEvent_t a, b;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_fail(e, "chert_fma_rate: events");
    e = cudaEventRecord(a, s);
    if (precision == CHERT_FP32)
        fma_chains_kernel<float><<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-7f);
    else
        fma_chains_kernel<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "chert_fma_rate: run");
    *flops_per_s = 2.0 * 8.0 * double(iters) * blocks * threads / (ms * 1e-3);
    return CHERT_OK;
}
