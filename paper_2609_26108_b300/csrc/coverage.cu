// Nodewise angular coverage of a 2D directional cache (the paper's angular-
// coverage validation, section "Nodewise local-truth and angular-coverage
// validation"): for every (mode, class) and stencil direction d = o/|o|,
//   * covered: two cyclically adjacent valid entries whose ray directions are
//     less than 90 degrees apart hold d on the closed short arc between them
//     (a bracket: the sampled ray-direction manifold passes through d);
//   * first-arrival branch: the bracket with the largest ray velocity
//     interpolated at d (V_e + t (V_e+1 - V_e), t = cross(r_e, d) /
//     cross(r_e, r_e+1)), ties to the lower e;
//   * branch mismatch: covered, and the entry the lookup of Eq. 27 picks
//     (largest d . r in the cache's precision, as chert_edge_table) is neither
//     end of that bracket -- at a fold (qSV cusp) the path search would take
//     a slower branch;
//   * missing angle: an entry valid in a reference cache of the same sampling
//     but flagged in this one.
// One warp per (mode, class); lanes take stencil directions, and every lane
// walks the class's entries (broadcast loads).  The bracket arithmetic is in
// double with every operation rounded separately, in a fixed order, so the
// counts are reproducible from the stored entries.
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace chert {
namespace {

constexpr int kCovMaxOff = 512;

struct CovOffsets {
    int n;
    short x[kCovMaxOff], z[kCovMaxOff];
};

__device__ __forceinline__ double cross2(double ax, double az, double bx, double bz) {
    return __dsub_rn(__dmul_rn(ax, bz), __dmul_rn(az, bx));
}
__device__ __forceinline__ double dot2(double ax, double az, double bx, double bz) {
    return __dadd_rn(__dmul_rn(ax, bx), __dmul_rn(az, bz));
}
__device__ __forceinline__ float lk_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double lk_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float lk_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double lk_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float lk_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double lk_div(double a, double b) { return __ddiv_rn(a, b); }

template <typename T>
__global__ void __launch_bounds__(256) coverage_kernel(const T* __restrict__ rx, const T* __restrict__ rz,
                                                       const T* __restrict__ V, const uint8_t* __restrict__ flag,
                                                       const uint8_t* __restrict__ truth, int n_mk, int n_dir,
                                                       CovOffsets off, int32_t* __restrict__ covered,
                                                       int32_t* __restrict__ mismatched,
                                                       int32_t* __restrict__ missing) {
    const int lane = threadIdx.x & 31;
    const long long w = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (w >= n_mk) return;
    const size_t base = static_cast<size_t>(w) * n_dir;
    int n_cov = 0, n_mis = 0;
    for (int o = lane; o < off.n; o += 32) {
        // d = o/|o| rounded as the lookup rounds it
        const double ox = off.x[o], oz = off.z[o];
        const T nrm = T(sqrt(ox * ox + oz * oz));
        const T tdx = lk_div(T(ox), nrm), tdz = lk_div(T(oz), nrm);
        const double dx = double(tdx), dz = double(tdz);
        // the lookup's pick (Eq. 27): first maximum of (dx*rx) + (dz*rz) in T
        T best = T(-INFINITY);
        int pick = -1;
        // the first-arrival bracket
        double vb = 0.0;
        int eb = -1;
        for (int e = 0; e < n_dir; ++e) {
            if (flag[base + e]) continue;
            const T rxe = rx[base + e], rze = rz[base + e];
            const T dt = lk_add(lk_mul(tdx, rxe), lk_mul(tdz, rze));
            if (dt > best) { best = dt; pick = e; }
            const int f = e + 1 == n_dir ? 0 : e + 1;
            if (flag[base + f]) continue;
            const double ax = double(rxe), az = double(rze);
            const double bx = double(rx[base + f]), bz = double(rz[base + f]);
            if (!(dot2(ax, az, bx, bz) > 0.0)) continue;
            const double c_ef = cross2(ax, az, bx, bz);
            const double c_ed = cross2(ax, az, dx, dz);
            const double c_df = cross2(dx, dz, bx, bz);
            bool inside;
            if (c_ef > 0.0) inside = c_ed >= 0.0 && c_df >= 0.0;
            else if (c_ef < 0.0) inside = c_ed <= 0.0 && c_df <= 0.0;
            else inside = c_ed == 0.0 && dot2(ax, az, dx, dz) > 0.0;
            if (!inside) continue;
            const double t = c_ef != 0.0 ? __ddiv_rn(c_ed, c_ef) : 0.0;
            const double ve = double(V[base + e]), vf = double(V[base + f]);
            const double v = __dadd_rn(ve, __dmul_rn(t, __dsub_rn(vf, ve)));
            if (eb < 0 || v > vb) { vb = v; eb = e; }
        }
        if (eb >= 0) {
            ++n_cov;
            const int fb = eb + 1 == n_dir ? 0 : eb + 1;
            if (pick != eb && pick != fb) ++n_mis;
        }
    }
    int n_miss = 0;
    if (truth)
        for (int e = lane; e < n_dir; e += 32) n_miss += (truth[base + e] == 0 && flag[base + e] != 0) ? 1 : 0;
    for (int s = 16; s > 0; s >>= 1) {
        n_cov += __shfl_xor_sync(0xffffffffu, n_cov, s);
        n_mis += __shfl_xor_sync(0xffffffffu, n_mis, s);
        n_miss += __shfl_xor_sync(0xffffffffu, n_miss, s);
    }
    if (lane == 0) {
        covered[w] = n_cov;
        mismatched[w] = n_mis;
        missing[w] = n_miss;
    }
}

}  // namespace
}  // namespace chert

extern "C" int chert_angular_coverage(const chert_cache_arrays* cache, int n_modes, int n_classes, int n_dir,
                                      int precision, const int32_t* offsets, int n_off,
                                      const uint8_t* d_truth_flag, int32_t* d_covered, int32_t* d_mismatched,
                                      int32_t* d_missing, void* stream) {
    using namespace chert;
    const char* who = "chert_angular_coverage";
    CHERT_REQUIRE(cache && cache->rx && cache->rz && cache->V && cache->flag && offsets && d_covered &&
                      d_mismatched && d_missing,
                  "%s: NULL argument", who);
    CHERT_REQUIRE(n_modes >= 1 && n_classes >= 1 && n_dir >= 2, "%s: counts", who);
    CHERT_REQUIRE(n_off >= 1 && n_off <= kCovMaxOff, "%s: n_off=%d (1..%d)", who, n_off, kCovMaxOff);
    CHERT_REQUIRE(precision == CHERT_FP64 || precision == CHERT_FP32 || precision == CHERT_MIXED,
                  "%s: precision=%d", who, precision);
    CovOffsets off{};
    off.n = n_off;
    for (int i = 0; i < n_off; ++i) {
        const int ox = offsets[3 * i], oy = offsets[3 * i + 1], oz = offsets[3 * i + 2];
        CHERT_REQUIRE(oy == 0, "%s: offset %d has oy=%d (2D caches only)", who, i, oy);
        CHERT_REQUIRE((ox || oz) && ox >= -32768 && ox <= 32767 && oz >= -32768 && oz <= 32767,
                      "%s: offset %d = (%d, %d)", who, i, ox, oz);
        off.x[i] = (short)ox;
        off.z[i] = (short)oz;
    }
    const long long n_mk = (long long)n_modes * n_classes;
    CHERT_REQUIRE(n_mk <= 0x7fffffffLL, "%s: problem too large", who);
    const unsigned blocks = (unsigned)((n_mk * 32 + 255) / 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == CHERT_FP64)
        coverage_kernel<double><<<blocks, 256, 0, s>>>(
            static_cast<const double*>(cache->rx), static_cast<const double*>(cache->rz),
            static_cast<const double*>(cache->V), cache->flag, d_truth_flag, (int)n_mk, n_dir, off, d_covered,
            d_mismatched, d_missing);
    else
        coverage_kernel<float><<<blocks, 256, 0, s>>>(
            static_cast<const float*>(cache->rx), static_cast<const float*>(cache->rz),
            static_cast<const float*>(cache->V), cache->flag, d_truth_flag, (int)n_mk, n_dir, off, d_covered,
            d_mismatched, d_missing);
    return launch_check(who);
}
