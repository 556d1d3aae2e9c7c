// Cache surrogate: an MLP per wave mode (7 -> 256 -> 256 -> 256 -> 256 -> 5,
// SiLU) that predicts the correction of one cache entry (the homogeneity
// solve of Eq. 9-11 at a folded slowness angle) to the exact elastic ray
// quantities of the same medium.  BF16 operands, FP32 accumulation and FP32
// master weights; all GEMMs have the form C = A * B^T with A [M x K] and
// B [N x K] row-major (K contiguous).
//
// Parameter vector (float, one per network), in this order:
//   W0 [256 x 7], b0 [256], W1..W3 [256 x 256], b1..b3 [256], W4 [5 x 256],
//   b4 [5], out_mean [5], out_std [5] (output standardisation, not trained).
//
// Inputs (features) are the folded slowness angle and the dimensionless
// medium (Vs0/Vp0, eps, delta, gamma, 1/Qp, 1/Qs) scaled to [-1, 1] over the
// training range; outputs, after un-standardising, are (V/Vg - 1, log(A/A0),
// psi - psi_el, validity logit, vartheta) with the attenuation learnt as a
// logarithm, where Vg and psi_el are the elastic group velocity and ray angle
// (closed form, derivative by hand) and A0 the attenuation of the homogeneous
// plane wave along the slowness direction, projected on the elastic ray.
#include <cuda_bf16.h>
#include <atomic>
#include <math.h>
#include <stdint.h>

#include "common.cuh"
#include "cplx.cuh"
#include "mlp_gemm.cuh"

namespace chert {
namespace mlp {

constexpr int kIn = 7, kInPad = 8, kHid = 256, kLayers = 4, kOut = 5;
__constant__ float kRangeLo[kIn] = {0.0f, 0.49f, 0.04f, -0.11f, 0.0f, 0.004f, 0.004f};
__constant__ float kRangeHi[kIn] = {1.5707963267948966f, 0.6f, 0.31f, 0.21f, 0.21f, 0.051f, 0.051f};

struct Layout {
    size_t W[kLayers + 1], b[kLayers + 1], mean, std, total;
};

__host__ __device__ inline Layout layout() {
    Layout L{};
    size_t o = 0;
    const int in[kLayers + 1] = {kIn, kHid, kHid, kHid, kHid};
    const int out[kLayers + 1] = {kHid, kHid, kHid, kHid, kOut};
    for (int l = 0; l <= kLayers; ++l) {
        L.W[l] = o; o += (size_t)in[l] * out[l];
        L.b[l] = o; o += out[l];
    }
    L.mean = o; o += kOut;
    L.std = o; o += kOut;
    L.total = o;
    return L;
}

// ----------------------------------------------------------------- features
struct MediumDims {
    float rs, eps, delta, gamma, iqp, iqs;   // dimensionless medium
    float a11, a13, a33, a44, a66;           // real moduli / Vp0^2
    float b11, b13, b33, b44, b66;           // imaginary moduli / Vp0^2 (a = aR - i aI)
};

// Dimensionless medium of a class: moduli over a33 (= Vp0^2); Thomsen's
// parameters and the two quality factors recovered from the stored moduli.
__device__ inline MediumDims dims_of(const chert_class& c) {
    MediumDims d;
    const double a33 = c.aR[2], a44 = c.aR[3];
    d.a11 = float(c.aR[0] / a33);
    d.a13 = float(c.aR[1] / a33);
    d.a33 = 1.0f;
    d.a44 = float(a44 / a33);
    d.a66 = float(c.aR[4] / a33);
    d.rs = float(sqrt(a44 / a33));
    d.eps = float((c.aR[0] - a33) / (2.0 * a33));
    d.gamma = float((c.aR[4] - a44) / (2.0 * a44));
    const double s = c.aR[1] + a44;
    d.delta = float((s * s - (a33 - a44) * (a33 - a44)) / (2.0 * a33 * (a33 - a44)));
    d.iqp = float(c.aI[2] / a33);
    d.iqs = float(c.aI[3] / a44);
    d.b11 = float(c.aI[0] / a33);
    d.b13 = float(c.aI[1] / a33);
    d.b33 = float(c.aI[2] / a33);
    d.b44 = float(c.aI[3] / a33);
    d.b66 = float(c.aI[4] / a33);
    return d;
}

// Attenuation baseline (in units of 1/Vp0): the homogeneous plane wave along the
// real slowness direction th has the complex phase velocity c = sqrt(lambda)
// of the complex Christoffel block, and decays by Im(1/c) per unit length along
// that direction; projected on the elastic ray direction psi_el.
__device__ inline float attenuation_baseline(const MediumDims& m, int mode, float th, float psi_el) {
    float s, c;
    sincosf(th, &s, &c);
    const float s2 = s * s, c2 = c * c;
    const cplx<float> a11 = mk(m.a11, -m.b11), a13 = mk(m.a13, -m.b13), a33 = mk(m.a33, -m.b33);
    const cplx<float> a44 = mk(m.a44, -m.b44), a66 = mk(m.a66, -m.b66);
    cplx<float> lam;
    if (mode == CHERT_QSH) {
        lam = s2 * a66 + c2 * a44;
    } else {
        const cplx<float> g11 = s2 * a11 + c2 * a44, g33 = s2 * a44 + c2 * a33;
        const cplx<float> g13 = (s * c) * (a13 + a44);
        const cplx<float> d = g11 - g33;
        const cplx<float> root = csqrt(d * d + 4.0f * (g13 * g13));
        const cplx<float> l1 = 0.5f * (g11 + g33 + root), l2 = 0.5f * (g11 + g33 - root);
        lam = ((mode == CHERT_QP) == (l1.re >= l2.re)) ? l1 : l2;
    }
    const cplx<float> inv = mk(1.0f, 0.0f) / csqrt(lam);
    return inv.im * cosf(psi_el - th);
}

// Elastic group velocity (in units of Vp0) and ray angle at slowness angle th.
__device__ inline void elastic_baseline(const MediumDims& m, int mode, float th, float& Vg, float& psi) {
    float s, c;
    sincosf(th, &s, &c);
    float lam, dlam;
    if (mode == CHERT_QSH) {
        lam = m.a66 * s * s + m.a44 * c * c;
        dlam = 2.0f * s * c * (m.a66 - m.a44);
    } else {
        const float b = m.a13 + m.a44;
        const float g11 = m.a11 * s * s + m.a44 * c * c, g33 = m.a44 * s * s + m.a33 * c * c;
        const float g13 = b * s * c;
        const float d11 = 2.0f * s * c * (m.a11 - m.a44), d33 = 2.0f * s * c * (m.a44 - m.a33);
        const float d13 = b * (c * c - s * s);
        const float D = (g11 - g33) * (g11 - g33) + 4.0f * g13 * g13;
        const float dD = 2.0f * (g11 - g33) * (d11 - d33) + 8.0f * g13 * d13;
        const float root = sqrtf(D);
        const float droot = root > 0.0f ? dD / (2.0f * root) : 0.0f;
        const float sg = mode == CHERT_QP ? 1.0f : -1.0f;
        lam = 0.5f * (g11 + g33 + sg * root);
        dlam = 0.5f * (d11 + d33 + sg * droot);
    }
    const float V = sqrtf(lam), dV = dlam / (2.0f * V);
    Vg = sqrtf(V * V + dV * dV);
    psi = th + atan2f(dV, V);
}

__device__ inline bool scale_features(const MediumDims& m, float th, float* x) {
    const float raw[kIn] = {th, m.rs, m.eps, m.delta, m.gamma, m.iqp, m.iqs};
    bool outside = false;
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
        x[i] = 2.0f * (raw[i] - kRangeLo[i]) / (kRangeHi[i] - kRangeLo[i]) - 1.0f;
        outside |= fabsf(x[i]) > 1.0f;
    }
    return outside;
}

// One item per (mode slot, class, folded angle j): features and baseline.
__global__ void features_kernel(const chert_class* __restrict__ classes, int n_classes, int M,
                                int mode, float* __restrict__ x, float* __restrict__ Vg,
                                float* __restrict__ psi, float* __restrict__ A0, uint8_t* __restrict__ outside) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = (long long)n_classes * (M + 1);
    if (i >= n) return;
    const int j = int(i % (M + 1)), k = int(i / (M + 1));
    const MediumDims m = dims_of(classes[k]);
    const float th = float((M_PI / 2 * j) / M);
    float f[kIn];
    outside[i] = scale_features(m, th, f);
#pragma unroll
    for (int q = 0; q < kIn; ++q) x[i * kInPad + q] = f[q];
    x[i * kInPad + kIn] = 0.0f;
    float vg, ps;
    elastic_baseline(m, mode, th, vg, ps);
    Vg[i] = vg;
    psi[i] = ps;
    A0[i] = attenuation_baseline(m, mode, th, ps);
}

// A network answer counts as sure when its validity logit is at least this far
// from 0 (p outside [0.1, 0.9]).
constexpr float kSureLogit = 2.2f;
// qSV entries whose imaginary angle exceeds 1 degree (cusp and triplication
// region, where the exact solution moves far from the homogeneous wave) go to
// the exact solver; the training set leaves out their ray quantities beyond
// twice that angle (NaN targets), which the network then never has to fit.
constexpr float kQsvBranchAngle = 0.0174533f;         // 1 deg: the default fallback angle
constexpr float kQsvTrainAngle = 2.0f * kQsvBranchAngle;
// qSV entries whose predicted imaginary angle exceeds this go to the exact
// solver (chert_set_surrogate_qsv_angle; process-wide; 0 sends every qSV
// entry the network calls valid to the exact solver).
std::atomic<float> g_qsv_branch_angle{kQsvBranchAngle};

// Training targets from an exact cache (float or double arrays): entry d = j
// of the first quadrant (d = M for j = M, mirrored in z), rotated back into
// the local frame; raw targets (V/Vg - 1, log(A/A0), psi - psi_el, valid,
// vartheta).  The attenuation is learnt as a logarithm so that the network
// cannot return a negative or zero one (a zero-cost edge for the attenuation
// traveltime).  qSV entries with |vartheta| > kQsvTrainAngle get NaN targets
// for the outputs 0-2.
template <typename TC>
__global__ void targets_kernel(const chert_class* __restrict__ classes, int n_classes, int M,
                               int mode, int mode_slot, const TC* __restrict__ V, const TC* __restrict__ A,
                               const TC* __restrict__ rx, const TC* __restrict__ rz,
                               const TC* __restrict__ vt, const uint8_t* __restrict__ flag,
                               const float* __restrict__ Vg, const float* __restrict__ psi_el,
                               const float* __restrict__ A0, float* __restrict__ t) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = (long long)n_classes * (M + 1);
    if (i >= n) return;
    const int j = int(i % (M + 1)), k = int(i / (M + 1));
    const size_t e = ((size_t)mode_slot * n_classes + k) * (4 * M) + j;   // d = j (j = M: quadrant 1)
    float* o = t + i * kOut;
    if (flag[e]) {
        o[0] = o[1] = o[2] = o[4] = 0.0f;
        o[3] = 0.0f;
        return;
    }
    const double a33 = classes[k].aR[2];
    const double vp0 = sqrt(a33);
    const double tl = classes[k].tilt;
    double ct, st;
    sincos(tl, &st, &ct);
    const double gx = double(rx[e]), gz = double(rz[e]);
    double lx = gx * ct - gz * st, lz = gx * st + gz * ct;             // undo Eq. 36
    double vtheta = double(vt[e]);
    if (j == M) { lz = -lz; vtheta = -vtheta; }                        // quadrant 1 mirror
    const double psi = atan2(lx, lz);
    const double vg = double(Vg[i]) * vp0;
    o[0] = float(double(V[e]) / vg - 1.0);
    o[1] = float(log(fmax(double(A[e]) * vp0, 1e-30) / fmax(double(A0[i]), 1e-30)));
    double dpsi = psi - double(psi_el[i]);
    dpsi = atan2(sin(dpsi), cos(dpsi));
    o[2] = float(dpsi);
    o[3] = 1.0f;
    o[4] = float(vtheta);
    if (mode == CHERT_QSV && fabs(vtheta) > double(kQsvTrainAngle)) o[0] = o[1] = o[2] = __int_as_float(0x7fc00000);
}

// ----------------------------------------------------------------- training pieces
__global__ void to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

// out[c][r] = in[r][c] for a rows x cols bf16 matrix (padded pitch in/out).
__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in, int rows, int cols,
                                      int ld_in, __nv_bfloat16* __restrict__ out, int ld_out) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int r = by + yy, c = bx + threadIdx.x;
        if (r < rows && c < cols) tile[yy][threadIdx.x] = in[(size_t)r * ld_in + c];
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int c = bx + yy, r = by + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * ld_out + r] = tile[threadIdx.x][yy];
    }
}

// dL/dy of the mean loss (masked squared error on standardised outputs 0,1,2,4
// and logistic loss on output 3); accumulates the summed loss.
__global__ void loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                 const float* __restrict__ mean, const float* __restrict__ std,
                                 long long n, float* __restrict__ g, __nv_bfloat16* __restrict__ gb,
                                 float* __restrict__ loss) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < n) {
        const bool valid = t[i * kOut + 3] > 0.5f;
        const float inv_n = 1.0f / float(n);
#pragma unroll
        for (int k = 0; k < kOut; ++k) {
            float gk;
            if (k == 3) {
                const float z = y[i * kOut + 3], tt = t[i * kOut + 3];
                const float p = 1.0f / (1.0f + expf(-z));
                l += fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))) - tt * z;
                gk = p - tt;
            } else {
                const float tk = t[i * kOut + k];
                const float d = (valid && !isnan(tk)) ? y[i * kOut + k] - (tk - mean[k]) / std[k] : 0.0f;
                l += 0.5f * d * d;
                gk = d;
            }
            gk *= inv_n;
            g[i * kOut + k] = gk;
            gb[i * kOut + k] = __float2bfloat16_rn(gk);
        }
    }
    // block reduction of the loss
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x < 32) {
        l = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (threadIdx.x == 0) atomicAdd(loss, l / float(n));
    }
}

// db[c] = sum_r g[r][c]
__global__ void colsum_kernel(const float* __restrict__ g, long long rows, int cols, float* __restrict__ db) {
    const int c = blockIdx.x;
    float s = 0.0f;
    for (long long r = threadIdx.x; r < rows; r += blockDim.x) s += g[r * cols + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) db[c] = s;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
}

// Decode network outputs into the mirrored, tilted cache entries (Eq. 36).
// Items i of one chunk cover classes k0 .. k0 + n_chunk - 1 of n_total.
// An entry is handed to the exact solver (flag 2) when its medium lies outside
// the training range, when the network is unsure whether a decaying root
// exists (|logit| < 2.2, i.e. 0.1 < p < 0.9), or, for qSV, when the predicted
// imaginary angle exceeds 1 deg -- the cusp and triplication region where the
// selected root switches branch.

template <typename TO>
__global__ void decode_kernel(const chert_class* __restrict__ classes, int n_total, int k0, int n_chunk,
                              int M, int mi, int mode, const float* __restrict__ y, const float* __restrict__ mean,
                              const float* __restrict__ std, const float* __restrict__ Vg,
                              const float* __restrict__ psi_el, const float* __restrict__ A0,
                              const uint8_t* __restrict__ outside, float qsv_angle, chert_cache_arrays out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = (long long)n_chunk * (M + 1);
    if (i >= n) return;
    const int j = int(i % (M + 1)), k = k0 + int(i / (M + 1));
    const int n_classes = n_total;
    const chert_class c = classes[k];
    const double vp0 = sqrt(c.aR[2]);
    float t[kOut];
#pragma unroll
    for (int q = 0; q < kOut; ++q) t[q] = y[i * kOut + q] * std[q] + mean[q];
    const float logit = y[i * kOut + 3];
    const bool unsure = fabsf(logit) < kSureLogit ||
                        (mode == CHERT_QSV && logit > 0.0f && !(fabsf(t[4]) <= qsv_angle));
    // a tensor-core GEMM that gave up left y unwritten: every solve then goes
    // to the exact solver
    const bool gemm_failed = *(volatile int*)&gemm::g_tc_error != 0;
    const uint8_t fl = (outside[i] || unsure || gemm_failed) ? 2 : (logit > 0.0f ? 0 : 1);
    const double V = double(Vg[i]) * vp0 * (1.0 + t[0]);
    // qSH: the homogeneous plane wave's attenuation A0 is the exact one (its
    // energy velocity is homogeneous at vartheta = 0 in a VTI medium), so the
    // network's correction is not applied
    const double A = (mode == CHERT_QSH ? double(A0[i]) : double(A0[i]) * exp(double(t[1]))) / vp0;
    const double psi = double(psi_el[i]) + t[2];
    const double vr = 1.0, vi = -A * V;                  // v_I / v_R = -A V
    const double Q = vi == 0.0 ? INFINITY : -(vr * vr - vi * vi) / (2.0 * vr * vi);
    const double rxl = sin(psi), rzl = cos(psi);
    double ct, st;
    sincos(c.tilt, &st, &ct);
    int cnt, d[4], sx[4], sz[4];
    if (j == 0) { cnt = 2; d[0] = 0; sx[0] = sz[0] = 1; d[1] = 2 * M; sx[1] = sz[1] = -1; }
    else if (j == M) { cnt = 2; d[0] = M; sx[0] = 1; sz[0] = -1; d[1] = 3 * M; sx[1] = -1; sz[1] = 1; }
    else {
        cnt = 4;
        d[0] = j; sx[0] = 1; sz[0] = 1;
        d[1] = 2 * M - j; sx[1] = 1; sz[1] = -1;
        d[2] = 2 * M + j; sx[2] = -1; sz[2] = -1;
        d[3] = 4 * M - j; sx[3] = -1; sz[3] = 1;
    }
    for (int q = 0; q < cnt; ++q) {
        const size_t e = ((size_t)mi * n_classes + k) * (4 * M) + d[q];
        const double lx = sx[q] * rxl, lz = sz[q] * rzl;
        if (out.theta) ((TO*)out.theta)[e] = TO((M_PI / 2 * d[q]) / M + c.tilt);
        out.flag[e] = fl;
        const bool ok = fl == 0;
        ((TO*)out.V)[e] = ok ? TO(V) : TO(NAN);
        ((TO*)out.rx)[e] = ok ? TO(lx * ct + lz * st) : TO(NAN);
        ((TO*)out.rz)[e] = ok ? TO(-lx * st + lz * ct) : TO(NAN);
        if (out.A) ((TO*)out.A)[e] = ok ? TO(fmax(A, 0.0)) : TO(NAN);
        if (out.Q) ((TO*)out.Q)[e] = ok ? TO(Q) : TO(NAN);
        if (out.vartheta) ((TO*)out.vartheta)[e] = ok ? TO(double(t[4]) * sx[q] * sz[q]) : TO(NAN);
    }
}

// ----------------------------------------------------------------- workspace
struct Ws {
    __nv_bfloat16* xb;       // [n][8]
    float* z[kLayers];       // [n][256] pre-activations
    __nv_bfloat16* h[kLayers];  // [n][256] activations
    float* y;                // [n][5]
    float* g;                // [n][256] gradient (fp32)
    __nv_bfloat16* gb;       // [n][256] gradient (bf16), ping
    __nv_bfloat16* gb2;      // [n][256] pong
    __nv_bfloat16* gT;       // [256][n]
    __nv_bfloat16* hT;       // [256][n]
    __nv_bfloat16* wT;       // [256][256]
    __nv_bfloat16* wb;       // bf16 weights (param layout)
    float* grad;             // [param total]
    float* loss;             // [1]
    size_t bytes;
};

inline size_t al(size_t x) { return (x + 255) & ~size_t(255); }

Ws ws_carve(unsigned char* base, long long n, bool training) {
    Ws w{};
    const Layout L = layout();
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base ? base + o : nullptr; o += al(bytes); return p; };
    w.xb = (__nv_bfloat16*)take((size_t)n * kInPad * 2);
    for (int l = 0; l < kLayers; ++l) {
        w.z[l] = (float*)take(training ? (size_t)n * kHid * 4 : 0);
        w.h[l] = (__nv_bfloat16*)take(training || l < 2 ? (size_t)n * kHid * 2 : 0);
    }
    w.y = (float*)take((size_t)n * kOut * 4);
    w.wb = (__nv_bfloat16*)take(L.total * 2);
    if (training) {
        w.g = (float*)take((size_t)n * kHid * 4);
        w.gb = (__nv_bfloat16*)take((size_t)n * kHid * 2);
        w.gb2 = (__nv_bfloat16*)take((size_t)n * kHid * 2);
        w.gT = (__nv_bfloat16*)take((size_t)n * kHid * 2);
        w.hT = (__nv_bfloat16*)take((size_t)n * kHid * 2);
        w.wT = (__nv_bfloat16*)take((size_t)kHid * kHid * 2);
        w.grad = (float*)take(L.total * 4);
        w.loss = (float*)take(4);
    }
    w.bytes = o;
    return w;
}

inline unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (unsigned)(b > (1 << 20) ? (1 << 20) : (b < 1 ? 1 : b));
}

// Forward through the network; keeps z (training) and h per layer.
int forward(const Ws& w, const float* params, long long n, bool training, cudaStream_t s) {
    const Layout L = layout();
    to_bf16_kernel<<<grid_for(L.total, 256), 256, 0, s>>>(params, w.wb, (long long)L.total);
    const __nv_bfloat16* a = w.xb;
    int K = kInPad;
    int lda = kInPad;
    for (int l = 0; l < kLayers; ++l) {
        __nv_bfloat16* hout = training ? w.h[l] : w.h[l & 1];
        gemm::Epilogue e{};
        e.bias = params + L.b[l];
        e.z_out = training ? w.z[l] : nullptr;
        e.h_out = hout;
        e.mode = gemm::kBiasSilu;
        // layer 0 weights are [256 x 7]; the GEMM reads K = 8 with a zero pad
        const int rc = gemm::nt(a, lda, w.wb + L.W[l], l == 0 ? kIn : kHid, (int)n, kHid,
                                l == 0 ? kIn : K, e, s);
        if (rc) return rc;
        a = hout;
        K = kHid;
        lda = kHid;
    }
    gemm::Epilogue e{};
    e.bias = params + L.b[kLayers];
    e.y_out = w.y;
    e.mode = gemm::kBias;
    return gemm::nt(a, kHid, w.wb + L.W[kLayers], kHid, (int)n, kOut, kHid, e, s);
}

}  // namespace mlp
}  // namespace chert

using namespace chert;
using namespace chert::mlp;

extern "C" size_t chert_mlp_param_count(void) { return layout().total; }

extern "C" double chert_set_surrogate_qsv_angle(double rad) {
    if (rad < 0) return g_qsv_branch_angle.load();
    return g_qsv_branch_angle.exchange((float)rad);
}

extern "C" long long chert_mlp_set_wait_limit(long long polls) {
    long long before = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&before, gemm::g_tc_wait_limit, sizeof(before));
    if (e != cudaSuccess) return cuda_fail(e, "chert_mlp_set_wait_limit");
    if (polls < 0) return before;
    e = cudaMemcpyToSymbol(gemm::g_tc_wait_limit, &polls, sizeof(polls));
    if (e != cudaSuccess) return cuda_fail(e, "chert_mlp_set_wait_limit");
    return before;
}

extern "C" int chert_mlp_check(void* stream) {
    return gemm::tc::check_and_clear(static_cast<cudaStream_t>(stream), "chert_mlp_check");
}

extern "C" int chert_mlp_set_tensor_cores(int enable) {
    const int before = gemm::tc::tensor_cores_enabled() ? 1 : 0;
    gemm::tc::tensor_cores_enabled() = enable != 0;
    return before;
}

extern "C" size_t chert_mlp_workspace_bytes(int64_t n, int training) {
    if (n < 1) return 0;
    return ws_carve(nullptr, n, training != 0).bytes;
}

// The forward pass enqueued on s, without reading the tensor-core status.
static int forward_enqueue(const float* d_params, const float* d_x, int64_t n, float* d_y, void* d_ws,
                           size_t ws_bytes, cudaStream_t s, const char* who) {
    CHERT_REQUIRE(d_params && d_x && d_y && d_ws && n >= 1, "%s: bad argument", who);
    const Ws w = ws_carve(static_cast<unsigned char*>(d_ws), n, false);
    if (ws_bytes < w.bytes) {
        set_error("%s: workspace %zu < %zu bytes", who, ws_bytes, w.bytes);
        return CHERT_ENOMEM;
    }
    to_bf16_kernel<<<grid_for(n * kInPad, 256), 256, 0, s>>>(d_x, w.xb, n * kInPad);
    int rc = forward(w, d_params, n, false, s);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(d_y, w.y, sizeof(float) * n * kOut, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return launch_check(who);
}

extern "C" int chert_mlp_forward(const float* d_params, const float* d_x, int64_t n, float* d_y,
                                 void* d_ws, size_t ws_bytes, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = forward_enqueue(d_params, d_x, n, d_y, d_ws, ws_bytes, s, "chert_mlp_forward");
    return rc ? rc : gemm::tc::check_and_clear(s, "chert_mlp_forward");
}

extern "C" int chert_mlp_train_step(float* d_params, float* d_m, float* d_v, int step, float lr,
                                    const float* d_x, const float* d_t, int64_t n, float* d_loss,
                                    float* d_grad_out, void* d_ws, size_t ws_bytes, void* stream) {
    CHERT_REQUIRE(d_params && d_m && d_v && d_x && d_t && d_ws && n >= 1 && step >= 1,
                  "chert_mlp_train_step: bad argument");
    const Ws w = ws_carve(static_cast<unsigned char*>(d_ws), n, true);
    if (ws_bytes < w.bytes) {
        set_error("chert_mlp_train_step: workspace %zu < %zu bytes", ws_bytes, w.bytes);
        return CHERT_ENOMEM;
    }
    const Layout L = layout();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    to_bf16_kernel<<<grid_for(n * kInPad, 256), 256, 0, s>>>(d_x, w.xb, n * kInPad);
    int rc = forward(w, d_params, n, true, s);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(w.loss, 0, 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "chert_mlp_train_step");
    // output layer gradient (uses w.g/w.gb as [n][5])
    loss_grad_kernel<<<grid_for(n, 256), 256, 0, s>>>(w.y, d_t, d_params + L.mean, d_params + L.std, n,
                                                      w.g, w.gb, w.loss);
    const dim3 tb(32, 8);
    int rows_out = kOut;
    __nv_bfloat16* gcur = w.gb;            // bf16 gradient of the current layer's output
    __nv_bfloat16* gnext = w.gb2;
    for (int l = kLayers; l >= 0; --l) {
        const int in = l == 0 ? kIn : kHid;
        const int ld_in = l == 0 ? kInPad : kHid;
        const __nv_bfloat16* hin = l == 0 ? w.xb : w.h[l - 1];
        // dW[l] = G^T * Hin: A = G^T [out x n], B = Hin^T [in x n]
        transpose_bf16_kernel<<<dim3((rows_out + 31) / 32, (unsigned)((n + 31) / 32)), tb, 0, s>>>(
            gcur, (int)n, rows_out, rows_out, w.gT, (int)n);
        transpose_bf16_kernel<<<dim3((in + 31) / 32, (unsigned)((n + 31) / 32)), tb, 0, s>>>(
            hin, (int)n, in, ld_in, w.hT, (int)n);
        gemm::Epilogue ew{};
        ew.y_out = w.grad + L.W[l];
        ew.mode = gemm::kPlain;
        rc = gemm::nt(w.gT, (int)n, w.hT, (int)n, rows_out, in, (int)n, ew, s);
        if (rc) return rc;
        colsum_kernel<<<rows_out, 256, 0, s>>>(w.g, n, rows_out, w.grad + L.b[l]);
        if (l == 0) break;
        // G[l-1] = (G * W[l]) o silu'(Z[l-1]): A = G [n x out], B = W^T [256 x out]
        transpose_bf16_kernel<<<dim3((in + 31) / 32, (rows_out + 31) / 32), tb, 0, s>>>(
            w.wb + L.W[l], rows_out, in, in, w.wT, rows_out);
        gemm::Epilogue eg{};
        eg.z_in = w.z[l - 1];
        eg.g_out = w.g;
        eg.h_out = gnext;
        eg.mode = gemm::kDsilu;
        rc = gemm::nt(gcur, rows_out, w.wT, rows_out, (int)n, kHid, rows_out, eg, s);
        if (rc) return rc;
        rows_out = kHid;
        __nv_bfloat16* t = gcur;
        gcur = gnext;
        gnext = t;
    }
    if (d_grad_out) {
        e = cudaMemcpyAsync(d_grad_out, w.grad, sizeof(float) * L.total, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "chert_mlp_train_step");
    }
    if (lr > 0.0f) {
        const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
        adam_kernel<<<grid_for(L.mean, 256), 256, 0, s>>>(d_params, w.grad, d_m, d_v, (long long)L.mean,
                                                         lr, c1, c2);
    }
    if (d_loss) {
        e = cudaMemcpyAsync(d_loss, w.loss, 4, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "chert_mlp_train_step");
    }
    rc = launch_check("chert_mlp_train_step");
    return rc ? rc : gemm::tc::check_and_clear(s, "chert_mlp_train_step");
}

extern "C" int chert_surrogate_dataset(const chert_class* d_classes, int n_classes, int M, int mode,
                                       int mode_slot, const chert_cache_arrays* exact, int precision,
                                       float* d_x, float* d_t, void* d_scratch, size_t scratch_bytes,
                                       void* stream) {
    CHERT_REQUIRE(d_classes && exact && d_x && d_t && d_scratch && n_classes >= 1 && M >= 1,
                  "chert_surrogate_dataset: bad argument");
    const long long n = (long long)n_classes * (M + 1);
    CHERT_REQUIRE(scratch_bytes >= (size_t)n * 13, "chert_surrogate_dataset: scratch too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* Vg = static_cast<float*>(d_scratch);
    float* psi = Vg + n;
    float* A0 = psi + n;
    uint8_t* outside = reinterpret_cast<uint8_t*>(A0 + n);
    features_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_classes, n_classes, M, mode, d_x, Vg, psi, A0, outside);
    if (precision == CHERT_FP64)
        targets_kernel<double><<<grid_for(n, 256), 256, 0, s>>>(
            d_classes, n_classes, M, mode, mode_slot, (const double*)exact->V, (const double*)exact->A,
            (const double*)exact->rx, (const double*)exact->rz, (const double*)exact->vartheta,
            exact->flag, Vg, psi, A0, d_t);
    else
        targets_kernel<float><<<grid_for(n, 256), 256, 0, s>>>(
            d_classes, n_classes, M, mode, mode_slot, (const float*)exact->V, (const float*)exact->A,
            (const float*)exact->rx, (const float*)exact->rz, (const float*)exact->vartheta,
            exact->flag, Vg, psi, A0, d_t);
    return launch_check("chert_surrogate_dataset");
}

// Classes per inference chunk: about 4M entries at a time.
static int chunk_classes(int n_classes, int M) {
    const long long per = (long long)(M + 1);
    long long c = (4LL << 20) / per;
    if (c < 1) c = 1;
    return (int)(c < n_classes ? c : n_classes);
}

extern "C" size_t chert_surrogate_cache_workspace_bytes(int n_classes, int M) {
    if (n_classes < 1 || M < 1) return 0;
    const long long n = (long long)chunk_classes(n_classes, M) * (M + 1);
    return al((size_t)n * kInPad * 4) + al((size_t)n * 13) + al((size_t)n * kOut * 4) +
           ws_carve(nullptr, n, false).bytes;
}

namespace chert {
// chert_surrogate_cache; `check` reads the tensor-core status at the end (one
// synchronisation of the stream).
int surrogate_cache(const float* const* d_params_per_mode, const chert_class* d_classes, int n_classes,
                    const int* modes, int n_modes, int M, int precision, const chert_cache_arrays* out,
                    void* d_ws, size_t ws_bytes, void* stream, bool check);
}

extern "C" int chert_surrogate_cache(const float* const* d_params_per_mode, const chert_class* d_classes,
                                     int n_classes, const int* modes, int n_modes, int M, int precision,
                                     const chert_cache_arrays* out, void* d_ws, size_t ws_bytes,
                                     void* stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs);
    if (e != cudaSuccess) return cuda_fail(e, "chert_surrogate_cache: capture status");
    return chert::surrogate_cache(d_params_per_mode, d_classes, n_classes, modes, n_modes, M, precision, out, d_ws,
                                  ws_bytes, stream, cs == cudaStreamCaptureStatusNone);
}

int chert::surrogate_cache(const float* const* d_params_per_mode, const chert_class* d_classes, int n_classes,
                           const int* modes, int n_modes, int M, int precision, const chert_cache_arrays* out,
                           void* d_ws, size_t ws_bytes, void* stream, bool check) {
    CHERT_REQUIRE(d_params_per_mode && d_classes && modes && out && d_ws, "chert_surrogate_cache: NULL");
    CHERT_REQUIRE(n_classes >= 1 && M >= 1 && n_modes >= 1 && n_modes <= 3, "chert_surrogate_cache: counts");
    CHERT_REQUIRE(out->V && out->rx && out->rz && out->flag, "chert_surrogate_cache: outputs");
    const size_t need = chert_surrogate_cache_workspace_bytes(n_classes, M);
    if (ws_bytes < need) {
        set_error("chert_surrogate_cache: workspace %zu < %zu bytes", ws_bytes, need);
        return CHERT_ENOMEM;
    }
    const int chunk = chunk_classes(n_classes, M);
    const long long nmax = (long long)chunk * (M + 1);
    unsigned char* p = static_cast<unsigned char*>(d_ws);
    float* x = (float*)p; p += al((size_t)nmax * kInPad * 4);
    float* Vg = (float*)p;
    float* psi = Vg + nmax;
    float* A0 = psi + nmax;
    uint8_t* outside = (uint8_t*)(A0 + nmax); p += al((size_t)nmax * 13);
    float* y = (float*)p; p += al((size_t)nmax * kOut * 4);
    const size_t rest = ws_bytes - (size_t)(p - (unsigned char*)d_ws);
    const Layout L = layout();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float qsv_angle = g_qsv_branch_angle.load();
    for (int mi = 0; mi < n_modes; ++mi) {
        CHERT_REQUIRE(d_params_per_mode[mi], "chert_surrogate_cache: NULL parameters");
        const float* prm = d_params_per_mode[mi];
        for (int k0 = 0; k0 < n_classes; k0 += chunk) {
            const int nc = chunk < n_classes - k0 ? chunk : n_classes - k0;
            const long long n = (long long)nc * (M + 1);
            features_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_classes + k0, nc, M, modes[mi], x, Vg, psi,
                                                              A0, outside);
            int rc = forward_enqueue(prm, x, n, y, p, rest, s, "chert_surrogate_cache");
            if (rc) return rc;
            if (precision == CHERT_FP64)
                decode_kernel<double><<<grid_for(n, 256), 256, 0, s>>>(d_classes, n_classes, k0, nc, M, mi,
                                                                      modes[mi], y,
                                                                      prm + L.mean, prm + L.std, Vg, psi,
                                                                      A0, outside, qsv_angle, *out);
            else
                decode_kernel<float><<<grid_for(n, 256), 256, 0, s>>>(d_classes, n_classes, k0, nc, M, mi,
                                                                     modes[mi], y,
                                                                     prm + L.mean, prm + L.std, Vg, psi,
                                                                     A0, outside, qsv_angle, *out);
        }
    }
    const int rc = launch_check("chert_surrogate_cache");
    return rc || !check ? rc : gemm::tc::check_and_clear(s, "chert_surrogate_cache");
}
