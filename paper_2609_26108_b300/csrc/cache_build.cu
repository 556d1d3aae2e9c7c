// Directional cache build: one warp per (mode, class, folded slowness angle).
//
// For the folded real slowness angle theta in [0, pi/2] (the 0-90 deg TI range
// of the cache, Eq. 26) the warp searches the imaginary angle vartheta that makes
// the complex energy velocity homogeneous (Eq. 9): it walks the grid
// vartheta_k = k*h outward from 0, 16 points per side per step (one per lane),
// finds sign changes of the residual with a ballot, polishes each candidate by
// 33-way subdivision (one point per lane per round) and keeps the first
// decaying root in order of |vartheta|.  Walking outward and stopping at the
// first acceptable root returns exactly the root a full scan of the grid
// would select.  The ray quantities of Eq. 10-11 are then written to the up to
// four mirrored entries of the full circle and rotated by the tilt (Eq. 36).
//
// Velocity kernels, for n = (sin(theta + i vartheta), 0, cos(theta + i vartheta))
// (Eq. 7) and the 2x2 x-z block of the Christoffel matrix (Eq. 4):
//   OEV (Eq. 12): v = a_ijkl p_l g_j g_k / (g.g).
//   MEV (Eq. 13-14): v = Gbar p + 1/2 g^H [Gamma(p) - I] dg/dp with Gbar
//     unsymmetrised and g^H g = 1.  Because g^H [Gamma(p) - I] removes the
//     eigenvector itself, the correction collapses to the antisymmetric part of
//     a_ijkl p_l g*_j g_k, i.e. for this block
//       v_x += 1/2 (a13 - a55) p_z w,  v_z -= 1/2 (a13 - a55) p_x w,
//       w = (g*_x g_z - g_x g*_z) / (g^H g).
//   qSH is polarised along y: v = (a66 p_x, a44 p_z) for both kernels.
#include <math.h>
#include <stdint.h>

#include "common.cuh"
#include "cplx.cuh"

namespace chert {
namespace {

constexpr double kAcceptTol = 1e-9;   // decaying when v_I <= kAcceptTol * v_R
constexpr double kPolishTol = 1e-14;  // rad

template <typename T>
struct Medium {
    cplx<T> a11, a13, a33, a44, a66;
};

template <typename T>
__device__ __forceinline__ Medium<T> load_medium(const chert_class& c) {
    Medium<T> m;
    m.a11 = mk<T>(T(c.aR[0]), T(-c.aI[0]));
    m.a13 = mk<T>(T(c.aR[1]), T(-c.aI[1]));
    m.a33 = mk<T>(T(c.aR[2]), T(-c.aI[2]));
    m.a44 = mk<T>(T(c.aR[3]), T(-c.aI[3]));
    m.a66 = mk<T>(T(c.aR[4]), T(-c.aI[4]));
    return m;
}

__device__ __forceinline__ float ch_(float x) { return coshf(x); }
__device__ __forceinline__ double ch_(double x) { return cosh(x); }
__device__ __forceinline__ float sh_(float x) { return sinhf(x); }
__device__ __forceinline__ double sh_(double x) { return sinh(x); }

// Complex energy velocity (x and z components) at slowness angle theta + i vt,
// with s = sin(theta), c = cos(theta).
template <typename T>
__device__ __forceinline__ void energy_velocity(const Medium<T>& m, T s, T c, T vt, int mode,
                                                int kernel, cplx<T>& v1, cplx<T>& v3) {
    const T chv = ch_(vt), shv = sh_(vt);
    const cplx<T> n1 = mk<T>(s * chv, c * shv);     // sin(theta + i vt)
    const cplx<T> n3 = mk<T>(c * chv, -s * shv);    // cos(theta + i vt)
    const cplx<T> n11 = n1 * n1, n33 = n3 * n3;
    if (mode == CHERT_QSH) {
        const cplx<T> cc = csqrt(m.a66 * n11 + m.a44 * n33);
        v1 = m.a66 * (n1 / cc);
        v3 = m.a44 * (n3 / cc);
        return;
    }
    const cplx<T> b = m.a13 + m.a44;
    const cplx<T> G11 = m.a11 * n11 + m.a44 * n33;
    const cplx<T> G33 = m.a44 * n11 + m.a33 * n33;
    const cplx<T> G13 = b * (n1 * n3);
    const cplx<T> tr = G11 + G33;
    const cplx<T> dG = G11 - G33;
    const cplx<T> D = csqrt(dG * dG + T(4) * (G13 * G13));
    const cplx<T> l1 = T(0.5) * (tr + D), l2 = T(0.5) * (tr - D);
    const bool first_is_p = l1.re >= l2.re;
    const cplx<T> lam = (mode == CHERT_QP) == first_is_p ? l1 : l2;
    const cplx<T> cc = csqrt(lam);
    const cplx<T> p1 = n1 / cc, p3 = n3 / cc;
    // eigenvector of the 2x2 block: the better conditioned of two forms
    const cplx<T> gA1 = G13, gA3 = lam - G11;
    const cplx<T> gB1 = lam - G33, gB3 = G13;
    const bool useA = norm2(gA1) + norm2(gA3) >= norm2(gB1) + norm2(gB3);
    const cplx<T> g1 = useA ? gA1 : gB1, g3 = useA ? gA3 : gB3;
    const cplx<T> g11 = g1 * g1, g33 = g3 * g3, g13 = g1 * g3;
    const cplx<T> bb = g11 + g33;
    v1 = (m.a11 * p1 * g11 + m.a44 * p1 * g33 + b * p3 * g13) / bb;
    v3 = (m.a44 * p3 * g11 + m.a33 * p3 * g33 + b * p1 * g13) / bb;
    if (kernel == CHERT_MEV) {
        const T hh = norm2(g1) + norm2(g3);
        const cplx<T> gg = conj(g1) * g3;              // w = 2i Im(g1* g3) / hh
        const cplx<T> w = mk<T>(T(0), T(2) * gg.im / hh);
        const cplx<T> e = T(0.5) * (m.a13 - m.a44) * w;
        v1 = v1 + e * p3;
        v3 = v3 - e * p1;
    }
}

// Sign-carrying residual: (v^R x v^I)_y; the oracle divides by |v^R|^2 > 0,
// which changes neither its sign nor its zeros.
template <typename T>
__device__ __forceinline__ T residual(const Medium<T>& m, T s, T c, T vt, int mode, int kernel) {
    cplx<T> v1, v3;
    energy_velocity(m, s, c, vt, mode, kernel, v1, v3);
    return v1.re * v3.im - v3.re * v1.im;
}

template <typename T>
struct RayQ {
    T V, A, Q, rx, rz;
    bool ok;
};

// Eq. 10-11 at a root.
template <typename T>
__device__ __forceinline__ RayQ<T> ray_quantities(const Medium<T>& m, T s, T c, T vt, int mode,
                                                  int kernel) {
    cplx<T> v1, v3;
    energy_velocity(m, s, c, vt, mode, kernel, v1, v3);
    RayQ<T> q;
    const T vr = hyp(v1.re, v3.re);
    q.rx = v1.re / vr;
    q.rz = v3.re / vr;
    const T vi = v1.im * q.rx + v3.im * q.rz;
    const T mag2 = vr * vr + vi * vi;
    q.V = mag2 / vr;
    q.A = fmax(-vi / mag2, T(0));
    q.Q = vi == T(0) ? T(INFINITY) : -(vr * vr - vi * vi) / (T(2) * vr * vi);
    q.ok = vi <= T(kAcceptTol) * vr;
    return q;
}

// 33-way subdivision of the bracket [lo, hi] (f(lo) has sign flo): every
// round each lane evaluates one interior point and the warp keeps the first
// sub-interval with a sign change.  All lanes return the same root.
template <typename T>
__device__ T polish(const Medium<T>& m, T s, T c, int mode, int kernel, T lo, T hi, T flo,
                    int lane) {
    for (int round = 0; round < 12; ++round) {
        const T width = hi - lo;
        if (!(width > T(kPolishTol))) break;
        if (width <= T(2) * (sizeof(T) == 4 ? T(1.2e-7) : T(2.3e-16)) * fmax(fabs(lo), fabs(hi)))
            break;
        const T x = lo + width * T(lane + 1) / T(33);
        const T fx = residual(m, s, c, x, mode, kernel);
        const bool chg = (fx == T(0)) || (signbit(fx) != signbit(flo));
        const unsigned mask = __ballot_sync(0xffffffffu, chg);
        if (mask == 0u) {
            lo = __shfl_sync(0xffffffffu, x, 31);
            flo = __shfl_sync(0xffffffffu, fx, 31);
            continue;
        }
        const int i = __ffs(mask) - 1;
        const T xi = __shfl_sync(0xffffffffu, x, i);
        const T fi = __shfl_sync(0xffffffffu, fx, i);
        const T xp = __shfl_sync(0xffffffffu, x, i > 0 ? i - 1 : 0);
        const T fp = __shfl_sync(0xffffffffu, fx, i > 0 ? i - 1 : 0);
        if (fi == T(0)) return xi;
        if (i > 0) {
            lo = xp;
            flo = fp;
        }
        hi = xi;
    }
    return T(0.5) * (lo + hi);
}

struct Outs {
    void *V, *A, *Q, *rx, *rz, *theta, *vartheta;
    uint8_t* flag;
};

struct ModeList {
    int m[3];
    int n;
};

template <typename TO>
__device__ __forceinline__ void put(void* p, size_t i, double v) {
    if (p) reinterpret_cast<TO*>(p)[i] = TO(v);
}

// TS: scan precision, TP: polish + ray-quantity precision, TO: storage.
template <typename TS, typename TP, typename TO>
__global__ void __launch_bounds__(256) cache_build_kernel(const chert_class* __restrict__ classes,
                                                          int n_classes, ModeList modes, int M,
                                                          double h, int K, int kernel, Outs out) {
    const int lane = threadIdx.x & 31;
    const long long warp = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int per = M + 1;
    const long long total = static_cast<long long>(modes.n) * n_classes * per;
    if (warp >= total) return;
    const int j = static_cast<int>(warp % per);
    const int k = static_cast<int>((warp / per) % n_classes);
    const int mi = static_cast<int>(warp / (static_cast<long long>(per) * n_classes));
    const int mode = modes.m[mi];
    const chert_class cls = classes[k];
    const Medium<TS> ms = load_medium<TS>(cls);
    const Medium<TP> mp = load_medium<TP>(cls);
    const double theta = (M_PI / 2 * j) / M;
    double sd, cd;
    sincos(theta, &sd, &cd);
    const TS ss = TS(sd), cs = TS(cd);
    const TP sp = TP(sd), cp = TP(cd);
    const bool mixed = sizeof(TS) != sizeof(TP);

    // ---- walk the grid outward from vartheta = 0 ----
    bool found = false;
    TP root = TP(0);
    const TS f0 = residual(ms, ss, cs, TS(0), mode, kernel);
    if (f0 == TS(0)) {
        const RayQ<TP> q = ray_quantities(mp, sp, cp, TP(0), mode, kernel);
        if (q.ok) found = true;
    }
    TS prev_pos = f0, prev_neg = f0;
    for (int base = 0; !found && base < K; base += 16) {
        const int kk = base + 1 + (lane & 15);
        const bool neg = lane >= 16;
        const bool valid = kk <= K;
        const double xk = (neg ? -static_cast<double>(kk) : static_cast<double>(kk)) * h;
        const TS f = valid ? residual(ms, ss, cs, TS(xk), mode, kernel) : TS(NAN);
        TS fprev = __shfl_up_sync(0xffffffffu, f, 1);
        if ((lane & 15) == 0) fprev = neg ? prev_neg : prev_pos;
        const bool br = valid && (fprev * f < TS(0));
        const bool zr = valid && (f == TS(0));
        unsigned bmask = __ballot_sync(0xffffffffu, br);
        unsigned zmask = __ballot_sync(0xffffffffu, zr);
        prev_pos = __shfl_sync(0xffffffffu, f, 15);
        prev_neg = __shfl_sync(0xffffffffu, f, 31);
        while (!found && (bmask | zmask)) {
            const unsigned any = (bmask | zmask);
            const int l = __ffs((any | (any >> 16)) & 0xffffu) - 1;
            const double kkl = static_cast<double>(base + 1 + l);
            // brackets at inner distance kk-1 (key 2kk-1), then zeros at kk (key 2kk)
            TP cand[2];
            bool cok[2] = {false, false};
            for (int side = 0; side < 2; ++side) {      // 0: negative, 1: positive
                const int ln = side ? l : 16 + l;
                if (!((bmask >> ln) & 1u)) continue;
                const TS fl = __shfl_sync(0xffffffffu, side ? fprev : f, ln);
                TP lo = side ? TP((kkl - 1.0) * h) : TP(-kkl * h);
                TP hi = side ? TP(kkl * h) : TP(-(kkl - 1.0) * h);
                TP flo = TP(fl);
                bool usable = true;
                if (mixed) {
                    // re-take the bracket signs in the polish precision; if the
                    // root sits within float noise of a grid point, step one cell
                    const TP h2 = TP(h);
                    TP xs = lo - h2 + TP(lane & 3) * h2;     // lo-h, lo, hi, hi+h
                    if (lane >= 4) xs = lo;
                    const TP fx = residual(mp, sp, cp, xs, mode, kernel);
                    const TP fa = __shfl_sync(0xffffffffu, fx, 0), fb = __shfl_sync(0xffffffffu, fx, 1);
                    const TP fc = __shfl_sync(0xffffffffu, fx, 2), fd = __shfl_sync(0xffffffffu, fx, 3);
                    if (fb * fc < TP(0)) {
                        flo = fb;
                    } else if (fb == TP(0) || fc == TP(0)) {
                        lo = hi = (fb == TP(0)) ? lo : hi;
                    } else if (fa * fb < TP(0)) {
                        hi = lo; lo = lo - h2; flo = fa;
                    } else if (fc * fd < TP(0)) {
                        lo = hi; hi = hi + h2; flo = fc;
                    } else {
                        usable = false;
                    }
                }
                if (!usable) continue;
                const TP r = (lo == hi) ? lo : polish(mp, sp, cp, mode, kernel, lo, hi, flo, lane);
                const RayQ<TP> q = ray_quantities(mp, sp, cp, r, mode, kernel);
                cand[side] = r;
                cok[side] = q.ok;
            }
            if (cok[0] || cok[1]) {
                found = true;
                if (cok[0] && cok[1]) root = (fabs(cand[1]) < fabs(cand[0])) ? cand[1] : cand[0];
                else root = cok[0] ? cand[0] : cand[1];
                break;
            }
            for (int side = 0; side < 2 && !found; ++side) {   // negative first
                const int ln = side ? l : 16 + l;
                if (!((zmask >> ln) & 1u)) continue;
                const TP r = side ? TP(kkl * h) : TP(-kkl * h);
                const RayQ<TP> q = ray_quantities(mp, sp, cp, r, mode, kernel);
                if (q.ok) { found = true; root = r; }
            }
            bmask &= ~((1u << l) | (1u << (16 + l)));
            zmask &= ~((1u << l) | (1u << (16 + l)));
        }
    }

    // ---- write the mirrored entries ----
    RayQ<TP> q{};
    if (found) q = ray_quantities(mp, sp, cp, root, mode, kernel);
    const int nd = 4 * M;
    int d[4], sxv[4], szv[4], cnt;
    if (j == 0) {
        cnt = 2; d[0] = 0; sxv[0] = 1; szv[0] = 1; d[1] = 2 * M; sxv[1] = -1; szv[1] = -1;
    } else if (j == M) {
        cnt = 2; d[0] = M; sxv[0] = 1; szv[0] = -1; d[1] = 3 * M; sxv[1] = -1; szv[1] = 1;
    } else {
        cnt = 4;
        d[0] = j;         sxv[0] = 1;  szv[0] = 1;
        d[1] = 2 * M - j; sxv[1] = 1;  szv[1] = -1;
        d[2] = 2 * M + j; sxv[2] = -1; szv[2] = -1;
        d[3] = 4 * M - j; sxv[3] = -1; szv[3] = 1;
    }
    if (lane < cnt) {
        const size_t e = (static_cast<size_t>(mi) * n_classes + k) * nd + d[lane];
        double ct, st;
        sincos(cls.tilt, &st, &ct);
        const double sx = sxv[lane], sz = szv[lane];
        put<TO>(out.theta, e, (M_PI / 2 * d[lane]) / M + cls.tilt);
        if (found) {
            const double lx = sx * double(q.rx), lz = sz * double(q.rz);
            put<TO>(out.rx, e, lx * ct + lz * st);
            put<TO>(out.rz, e, -lx * st + lz * ct);
            put<TO>(out.V, e, double(q.V));
            put<TO>(out.A, e, double(q.A));
            put<TO>(out.Q, e, double(q.Q));
            put<TO>(out.vartheta, e, double(root) * sx * sz);
            out.flag[e] = 0;
        } else {
            put<TO>(out.rx, e, NAN);
            put<TO>(out.rz, e, NAN);
            put<TO>(out.V, e, NAN);
            put<TO>(out.A, e, NAN);
            put<TO>(out.Q, e, NAN);
            put<TO>(out.vartheta, e, NAN);
            out.flag[e] = 1;
        }
    }
}

}  // namespace
}  // namespace chert

extern "C" int chert_build_cache(const chert_class* d_classes, int n_classes, const int* modes,
                                 int n_modes, const chert_cache_params* params,
                                 const chert_cache_arrays* out, void* stream) {
    using namespace chert;
    CHERT_REQUIRE(d_classes && modes && params && out, "chert_build_cache: NULL argument");
    CHERT_REQUIRE(n_classes >= 1, "chert_build_cache: n_classes=%d", n_classes);
    CHERT_REQUIRE(n_modes >= 1 && n_modes <= 3, "chert_build_cache: n_modes=%d", n_modes);
    CHERT_REQUIRE(params->M >= 1 && params->M <= (1 << 20), "chert_build_cache: M=%d", params->M);
    CHERT_REQUIRE(params->scan_step > 0 && params->scan_half >= 1 &&
                      params->scan_half <= (1 << 28),
                  "chert_build_cache: bad scan grid");
    CHERT_REQUIRE(params->kernel == CHERT_OEV || params->kernel == CHERT_MEV,
                  "chert_build_cache: kernel=%d", params->kernel);
    CHERT_REQUIRE(out->V && out->rx && out->rz && out->flag,
                  "chert_build_cache: V, rx, rz and flag outputs are required");
    ModeList ml{{0, 0, 0}, n_modes};
    for (int i = 0; i < n_modes; i++) {
        CHERT_REQUIRE(modes[i] >= CHERT_QP && modes[i] <= CHERT_QSH, "chert_build_cache: mode %d",
                      modes[i]);
        for (int j = 0; j < i; j++)
            CHERT_REQUIRE(modes[j] != modes[i], "chert_build_cache: repeated mode");
        ml.m[i] = modes[i];
    }
    Outs o{out->V, out->A, out->Q, out->rx, out->rz, out->theta, out->vartheta, out->flag};
    const long long warps = static_cast<long long>(n_modes) * n_classes * (params->M + 1);
    const int threads = 256;
    const long long blocks = (warps * 32 + threads - 1) / threads;
    CHERT_REQUIRE(blocks < (1LL << 31), "chert_build_cache: problem too large");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double h = params->scan_step;
    const int K = params->scan_half;
    switch (params->precision) {
        case CHERT_FP64:
            cache_build_kernel<double, double, double><<<(unsigned)blocks, threads, 0, s>>>(
                d_classes, n_classes, ml, params->M, h, K, params->kernel, o);
            break;
        case CHERT_FP32:
            cache_build_kernel<float, float, float><<<(unsigned)blocks, threads, 0, s>>>(
                d_classes, n_classes, ml, params->M, h, K, params->kernel, o);
            break;
        case CHERT_MIXED:
            cache_build_kernel<float, double, float><<<(unsigned)blocks, threads, 0, s>>>(
                d_classes, n_classes, ml, params->M, h, K, params->kernel, o);
            break;
        default:
            CHERT_REQUIRE(false, "chert_build_cache: precision=%d", params->precision);
    }
    return launch_check("chert_build_cache");
}
