// Directional cache build: one warp per (mode, class, folded slowness angle),
// and a second launch that gives the few solves with a far (or no) root a
// whole CTA.
//
// For the folded real slowness angle theta in [0, pi/2] (the 0-90 deg TI range
// of the cache, Eq. 26) the warp searches the imaginary angle vartheta that makes
// the complex energy velocity homogeneous (Eq. 9): it walks the grid
// vartheta_k = k*h outward from 0, 64 points per side per step (4 per lane),
// finds sign changes of the residual with a ballot, polishes each candidate by
// 33-way subdivision (one point per lane per round) and keeps the first
// decaying root in order of |vartheta|.  Walking outward and stopping at the
// first acceptable root returns exactly the root a full scan of the grid
// would select.  The ray quantities of Eq. 10-11 are then written to the up to
// four mirrored entries of the full circle and rotated by the tilt (Eq. 36).
// In 3D (chert_build_cache_3d) each global slowness direction is one solve in
// the sagittal plane of the class's symmetry-axis frame (Eq. 35), and its ray
// is turned back to the global frame.  Precisions: FP64 (all double), FP32
// (all float) and MIXED (float scan and polish, then a float-float refinement
// of the accepted root and its ray quantities, float storage).
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

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "cplx.cuh"
#include "ff.cuh"

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

__device__ __forceinline__ float shfl(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Relative precision of each arithmetic (float, float-float, double).
template <typename T>
constexpr double unit_eps();
template <>
constexpr double unit_eps<float>() { return 1.2e-7; }
template <>
constexpr double unit_eps<xf::ff>() { return 3.6e-15; }
template <>
constexpr double unit_eps<double>() { return 2.3e-16; }

__device__ __forceinline__ float ch_(float x) { return coshf(x); }
__device__ __forceinline__ double ch_(double x) { return cosh(x); }
__device__ __forceinline__ float sh_(float x) { return sinhf(x); }
__device__ __forceinline__ double sh_(double x) { return sinh(x); }

// Complex energy velocity (x and z components) at slowness angle theta + i vt,
// with s = sin(theta), c = cos(theta).  If cond is not null it receives the
// squared amplification of rounding errors in v: (|tr|/|D|)^2 (the eigen-gap
// of the 2x2 block, tr its trace, D the square root of its discriminant) times
// (|g|^2/|g.g|)^2 (the bilinear norm that divides v), 1 for qSH, and +inf
// where the qP/qSV labels are ambiguous (Re D within 2^-14 |tr| of 0: the two
// eigenvalues' real parts, which order the labels, nearly coincide).
template <typename T>
__device__ __forceinline__ void energy_velocity_body(const Medium<T>& m, T s, T c, T vt, int mode,
                                                     int kernel, cplx<T>& v1, cplx<T>& v3, bool want_cond,
                                                     T& cond) {
    const T chv = ch_(vt), shv = sh_(vt);
    const cplx<T> n1 = mk<T>(s * chv, c * shv);     // sin(theta + i vt)
    const cplx<T> n3 = mk<T>(c * chv, -s * shv);    // cos(theta + i vt)
    const cplx<T> n11 = n1 * n1, n33 = n3 * n3;
    if (mode == CHERT_QSH) {
        const cplx<T> cc = csqrt(m.a66 * n11 + m.a44 * n33);
        v1 = m.a66 * (n1 / cc);
        v3 = m.a44 * (n3 / cc);
        cond = T(1);
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
    cond = T(1);
    if (want_cond) {
        const T trn = norm2(tr);
        if (D.re * D.re < T(0x1p-28) * trn) {
            cond = T(INFINITY);
        } else {
            const T hh = norm2(g1) + norm2(g3);
            cond = (trn / norm2(D)) * (hh * hh / norm2(bb));
        }
    }
}

// One out-of-line copy of the evaluation, per precision, serves every call
// site (the scan's grid points, the polish, the refinement, the ray
// quantities).  Inlined, the scan loop alone held four copies and the kernel
// stalled on instruction fetch (ncu: ~16 cycles of "no instruction" per issue
// on the per-cell builds); out of line, the per-cell qP and qSV builds run
// 26% and 17% faster.  The medium goes in and the velocities come out by
// value, so the call passes them in registers rather than through a stack
// frame in local memory.
template <typename T>
struct EnergyVelocity {
    cplx<T> v1, v3;
    T cond;
};

// Evaluation counter (instrumentation, off by default): evaluations of the
// energy velocity in float, float-float and double, one per thread and call.
__device__ int g_eval_count_on = 0;
__device__ unsigned long long g_eval_count[3] = {0, 0, 0};

template <typename T>
__device__ __forceinline__ void count_eval() {
    if (g_eval_count_on) {
        const unsigned active = __activemask();
        if ((threadIdx.x & 31) == __ffs(active) - 1)
            atomicAdd(&g_eval_count[sizeof(T) == 4 ? 0 : (sizeof(T) == 8 && !std::is_same<T, double>::value) ? 1 : 2],
                      (unsigned long long)__popc(active));
    }
}

template <typename T>
__device__ __noinline__ EnergyVelocity<T> energy_velocity_val(Medium<T> m, T s, T c, T vt, int mode, int kernel,
                                                              bool want_cond) {
    count_eval<T>();
    EnergyVelocity<T> r;
    energy_velocity_body(m, s, c, vt, mode, kernel, r.v1, r.v3, want_cond, r.cond);
    return r;
}
template <typename T>
__device__ __forceinline__ void energy_velocity_call(const Medium<T>& m, T s, T c, T vt, int mode, int kernel,
                                                     cplx<T>& v1, cplx<T>& v3, T* cond = nullptr) {
    const EnergyVelocity<T> r = energy_velocity_val(m, s, c, vt, mode, kernel, cond != nullptr);
    v1 = r.v1;
    v3 = r.v3;
    if (cond) *cond = r.cond;
}
template <typename T>
__device__ __forceinline__ void energy_velocity(const Medium<T>& m, T s, T c, T vt, int mode,
                                                int kernel, cplx<T>& v1, cplx<T>& v3) {
    energy_velocity_call(m, s, c, vt, mode, kernel, v1, v3);
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
__device__ __forceinline__ T residual_cold(const Medium<T>& m, T s, T c, T vt, int mode, int kernel) {
    cplx<T> v1, v3;
    energy_velocity_call(m, s, c, vt, mode, kernel, v1, v3);
    return v1.re * v3.im - v3.re * v1.im;
}

// Noise guard of the MIXED scan.  The float residual's rounding error,
// measured against float-float evaluations over the whole [-30, 30] deg grid
// of 1,008 media (the layered benchmark's and 1,000 per-cell ones), stays
// below 2.7e-7 (qP), 1.1e-6 (qSV) and 4.8e-7 (qSH) times kappa |v|^2
// (kappa^2 = the cond factor of energy_velocity_body).  A float sign is
// trusted only where |f| >= G kappa |v|^2 with G = 2^-18, 2^-16 and 2^-17 for
// the three modes, a margin of about 14 over that noise; below it (under
// 1e-4 of the grid points) the sign is taken from a float-float evaluation
// at the exact grid point k*h, which is what a double scan sees.
__device__ __forceinline__ float guard2(int mode) {
    return mode == CHERT_QP ? 0x1p-36f : mode == CHERT_QSV ? 0x1p-32f : 0x1p-34f;   // G^2
}

// Float residual with its guard: returns f; need = whether |f| is within the
// guard of zero (or the mode labels are ambiguous).
__device__ __forceinline__ float residual_guarded(const Medium<float>& m, float s, float c, float vt, int mode,
                                                  int kernel, bool& need) {
    cplx<float> v1, v3;
    float cond;
    energy_velocity_call(m, s, c, vt, mode, kernel, v1, v3, &cond);
    const float f = v1.re * v3.im - v3.re * v1.im;
    const float sc = norm2(v1) + norm2(v3);
    need = !(f * f >= guard2(mode) * cond * (sc * sc));    // NaN or inf bounds also re-evaluate
    return f;
}

// A residual of the refinement precision narrowed to the scan precision with
// its sign kept (0 only for an exact zero).
template <typename TP>
__device__ __forceinline__ float narrow_sign(TP r) {
    const double d = double(r);
    if (d == 0.0) return 0.0f;
    const float f = float(d);
    return f != 0.0f ? f : copysignf(1.17549435e-38f, float(d > 0.0 ? 1 : -1));
}

template <typename T>
struct RayQ {
    T V, A, Q, rx, rz, vr, vi;
    bool ok;
};

// Eq. 10-11 from the complex energy velocity at a root.
template <typename T>
__device__ __forceinline__ RayQ<T> ray_from_velocity(cplx<T> v1, cplx<T> v3) {
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
    q.vr = vr;
    q.vi = vi;
    return q;
}

template <typename T>
__device__ __forceinline__ RayQ<T> ray_quantities(const Medium<T>& m, T s, T c, T vt, int mode,
                                                  int kernel) {
    cplx<T> v1, v3;
    energy_velocity_call(m, s, c, vt, mode, kernel, v1, v3);
    return ray_from_velocity(v1, v3);
}

// 33-way subdivision of the bracket [lo, hi] (residuals flo, fhi at its ends):
// every round each lane evaluates one interior point and the warp keeps the
// first sub-interval with a sign change, until the bracket is narrower than
// `stop` or than the precision allows; a final secant step inside the last
// bracket then places the root (its error is of the order of the squared
// bracket width).  All lanes return the same root.
template <typename T>
__device__ T polish(const Medium<T>& m, T s, T c, int mode, int kernel, T lo, T hi, T flo, T fhi,
                    int lane, T stop) {
    constexpr T eps = T(unit_eps<T>());
    for (int round = 0; round < 12; ++round) {
        const T width = hi - lo;
        if (!(width > stop) || !(width > T(kPolishTol))) break;
        if (width <= T(2) * eps * fmax(fabs(lo), fabs(hi))) break;
        const T x = lo + width * T(lane + 1) / T(33);
        const T fx = residual_cold(m, s, c, x, mode, kernel);
        const bool chg = (fx == T(0)) || (signbit(fx) != signbit(flo));
        const unsigned mask = __ballot_sync(0xffffffffu, chg);
        if (mask == 0u) {
            lo = shfl(x, 31);
            flo = shfl(fx, 31);
            continue;
        }
        const int i = __ffs(mask) - 1;
        const T xi = shfl(x, i);
        const T fi = shfl(fx, i);
        const T xp = shfl(x, i > 0 ? i - 1 : 0);
        const T fp = shfl(fx, i > 0 ? i - 1 : 0);
        if (fi == T(0)) return xi;
        if (i > 0) {
            lo = xp;
            flo = fp;
        }
        hi = xi;
        fhi = fi;
    }
    if (flo != fhi && isfinite(flo) && isfinite(fhi)) {
        const T r = lo - flo * (hi - lo) / (fhi - flo);
        if (r >= lo && r <= hi) return r;
    }
    return T(0.5) * (lo + hi);
}

template <typename TP>
struct Refined {
    TP root;
    RayQ<TP> q;
};

template <typename T>
__device__ __forceinline__ cplx<T> shfl_c(cplx<T> v, int src) { return mk<T>(shfl(v.re, src), shfl(v.im, src)); }

// Extended-precision refinement (TP: float-float or double) of a float root
// r32 that lies in the grid bracket [glo, ghi] of width h.  The float root
// can be off by the float noise of the residual (it matters most for roots
// near vartheta = 0), so the window is [r32 - d, r32 + d] with d a quarter of
// h (at least 16 float ulps of r32), clipped to the bracket: one 32-point
// round (lanes 0 and 31 at the ends), a secant step between the two lanes
// around the sign change, and the ray quantities (Eq. 10-11) from the energy
// velocity interpolated linearly between those lanes (spacing h/62, so the
// interpolation error, of the order of its square, lies far below the
// precision of the stored float entries).  If the window shows no sign
// change, the whole bracket is polished in TP and evaluated there.  Out of
// line: called once per candidate that passes the float prefilter.
template <typename TP>
__device__ __noinline__ Refined<TP> refine(const Medium<TP>& m, TP s, TP c, int mode, int kernel, TP r32,
                                           TP glo, TP ghi, int lane) {
    const TP d = fmax(TP(0.25f) * (ghi - glo), TP(1e-8) + TP(16.0 * 1.2e-7) * fabs(r32));
    const TP a = fmax(glo, r32 - d), b = fmin(ghi, r32 + d);
    const TP x = a + (b - a) * TP(float(lane) / 31.0f);           // lane 0: a, lane 31: b
    cplx<TP> v1, v3;
    energy_velocity_call(m, s, c, x, mode, kernel, v1, v3);
    const TP fx = v1.re * v3.im - v3.re * v1.im;
    const TP fa = shfl(fx, 0), fb = shfl(fx, 31);
    Refined<TP> out;
    auto at_lane = [&](int l) {
        out.root = shfl(x, l);
        out.q = ray_from_velocity(shfl_c(v1, l), shfl_c(v3, l));
        return out;
    };
    if (fa == TP(0)) return at_lane(0);
    if (fb == TP(0)) return at_lane(31);
    if (signbit(fa) == signbit(fb)) {
        const TP flo = residual_cold(m, s, c, glo, mode, kernel);
        const TP fhi = residual_cold(m, s, c, ghi, mode, kernel);
        TP r;
        if (flo == TP(0)) r = glo;
        else if (fhi == TP(0)) r = ghi;
        else if (signbit(flo) == signbit(fhi)) r = r32;       // no sign change in TP: keep the float root
        else r = polish(m, s, c, mode, kernel, glo, ghi, flo, fhi, lane, TP(1e-9));
        out.root = r;
        out.q = ray_quantities(m, s, c, r, mode, kernel);
        return out;
    }
    const bool chg = (fx == TP(0)) || (signbit(fx) != signbit(fa));
    const unsigned mask = __ballot_sync(0xffffffffu, chg) & ~1u;
    const int i = __ffs(mask) - 1;                             // first lane past a sign change
    const TP xi = shfl(x, i), fi = shfl(fx, i);
    const TP xp = shfl(x, i - 1), fp = shfl(fx, i - 1);
    if (fi == TP(0)) return at_lane(i);
    TP r = xp - fp * (xi - xp) / (fi - fp);
    if (!(r >= xp && r <= xi)) r = TP(0.5f) * (xp + xi);
    const TP t = (r - xp) / (xi - xp);
    const cplx<TP> a1 = shfl_c(v1, i - 1), b1 = shfl_c(v1, i), a3 = shfl_c(v3, i - 1), b3 = shfl_c(v3, i);
    out.root = r;
    out.q = ray_from_velocity(a1 + t * (b1 - a1), a3 + t * (b3 - a3));
    return out;
}

struct Outs {
    void *V, *A, *Q, *rx, *rz, *theta, *vartheta;
    uint8_t* flag;
    void *ry, *phi;          // 3D only
};

// Direction set of a cache.  2D (n_az == 0): 4M slowness angles of the local
// frame, solved as the M+1 folded angles j and mirrored.  3D (n_az > 0): the
// global directions of polar angle (i + 1/2) pi/n_pol and azimuth
// j 2 pi/n_az, entry d = i*n_az + j, one solve each (Eq. 35).
struct Geo {
    int M, n_az, n_pol;
    __host__ __device__ bool three_d() const { return n_az > 0; }
    __host__ __device__ int per_class() const { return n_az > 0 ? n_az * n_pol : M + 1; }   // solves
    __host__ __device__ int n_dir() const { return n_az > 0 ? n_az * n_pol : 4 * M; }       // entries
};

struct ModeList {
    int m[3];
    int n;
};

template <typename TO>
__device__ __forceinline__ void put(void* p, size_t i, double v) {
    if (p) reinterpret_cast<TO*>(p)[i] = TO(v);
}

constexpr int kPending = 2;          // flag value between the two launches
constexpr int kPhase1Reach = 2048;   // grid points per side scanned by the first launch

// One solve: (mode, class, folded angle index j), its medium and angle.
template <typename TS, typename TP>
struct Solve {
    int mi, k, j, mode;
    double sz, phl;          // 3D: mirror sign of the local polar angle, local azimuth
    chert_class cls;
    Medium<TS> ms;
    Medium<TP> mp;
    double sd, cd;
    TS ss, cs;
    TP sp, cp;
};

// Local frame of Eq. 35: rows e_x', e_y', e_z' of the symmetry axis (theta0, phi0).
__device__ __forceinline__ void local_basis(double theta0, double phi0, double E[3][3]) {
    double st, ct, sp, cp;
    sincos(theta0, &st, &ct);
    sincos(phi0, &sp, &cp);
    E[0][0] = ct * cp; E[0][1] = ct * sp; E[0][2] = -st;
    E[1][0] = -sp;     E[1][1] = cp;      E[1][2] = 0.0;
    E[2][0] = st * cp; E[2][1] = st * sp; E[2][2] = ct;
}

// 3D direction d of the global grid: polar and azimuth angles and unit vector.
__device__ __forceinline__ void global_direction(const Geo& g, int d, double& th, double& ph, double n[3]) {
    const int i = d / g.n_az, j = d % g.n_az;
    th = (i + 0.5) * M_PI / g.n_pol;
    ph = j * 2.0 * M_PI / g.n_az;
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    n[0] = st * cp; n[1] = st * sp; n[2] = ct;
}

template <typename TS, typename TP>
__device__ __forceinline__ Solve<TS, TP> make_solve(const chert_class* classes, int n_classes,
                                                     const ModeList& modes, const Geo& g, long long idx) {
    Solve<TS, TP> v;
    const int per = g.per_class();
    v.j = static_cast<int>(idx % per);
    v.k = static_cast<int>((idx / per) % n_classes);
    v.mi = static_cast<int>(idx / (static_cast<long long>(per) * n_classes));
    v.mode = modes.m[v.mi];
    v.cls = classes[v.k];
    v.ms = load_medium<TS>(v.cls);
    v.mp = load_medium<TP>(v.cls);
    v.sz = 1.0;
    v.phl = 0.0;
    double theta;
    if (g.three_d()) {
        // the sagittal-plane solve at the local polar angle folded into [0, pi/2]
        double th, ph, n[3], E[3][3];
        global_direction(g, v.j, th, ph, n);
        local_basis(v.cls.tilt, v.cls.azim, E);
        double nl[3];
        for (int r = 0; r < 3; ++r) nl[r] = E[r][0] * n[0] + E[r][1] * n[1] + E[r][2] * n[2];
        const double thl = acos(fmin(1.0, fmax(-1.0, nl[2])));
        v.phl = atan2(nl[1], nl[0]);
        v.sz = thl <= M_PI / 2 ? 1.0 : -1.0;
        theta = v.sz > 0 ? thl : M_PI - thl;
    } else {
        theta = (M_PI / 2 * v.j) / g.M;
    }
    sincos(theta, &v.sd, &v.cd);
    v.ss = TS(v.sd); v.cs = TS(v.cd);
    v.sp = TP(v.sd); v.cp = TP(v.cd);
    return v;
}

// Grid point kk*h in the scan precision.  In float it is formed from the
// two-float split h = hf + hl (hf = float(h), hl = float(h - hf)) as
// fma(kk, hf, kk*hl): one rounding of kk*h (kk < 2^24 is exact in float) and
// no double-precision instruction, which on this part issues at a small
// fraction of the float rate.
__device__ __forceinline__ float grid_point(float kf, double, float hf, float hl) {
    return fmaf(kf, hf, kf * hl);
}
__device__ __forceinline__ double grid_point(double kf, double h, float, float) { return kf * h; }

// Re-evaluation of the guarded grid points of one scan step in the
// refinement precision: the P points of lane l lie at grid distance
// base + 1 + (l & 15)*P + p, on the negative side for l >= 16.  The pending
// points of the whole warp are dealt out one per lane, so a step costs one
// refinement-precision evaluation per 32 pending points.
template <typename TP, typename TS, typename TSolve, int P>
__device__ __forceinline__ void guard_points(const TSolve& v, int kernel, double h, int base, TS (&fv)[P],
                                             const bool (&need)[P], int lane) {
    unsigned pm[P];
    int cum[P + 1];
    cum[0] = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        pm[p] = __ballot_sync(0xffffffffu, need[p]);
        cum[p + 1] = cum[p] + __popc(pm[p]);
    }
    const int total = cum[P];
    for (int first = 0; first < total; first += 32) {
        const int t = first + lane;
        TS r = TS(0);
        if (t < total) {
            int p = 0;
            while (t >= cum[p + 1]) ++p;
            unsigned m = pm[p];
            for (int i = cum[p]; i < t; ++i) m &= m - 1;          // drop the set bits before item t
            const int l = __ffs(m) - 1;
            const int kk = base + 1 + (l & 15) * P + p;
            const double x = (l >= 16 ? -1.0 : 1.0) * (double(kk) * h);
            r = narrow_sign(residual_cold(v.mp, v.sp, v.cp, TP(x), v.mode, kernel));
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int src = cum[p] + __popc(pm[p] & ((1u << lane) - 1u)) - first;
            const TS got = __shfl_sync(0xffffffffu, r, src & 31);
            if (need[p] && src >= 0 && src < 32) fv[p] = got;
        }
    }
}

// The residual at one grid distance kk (>= 0) on side sgn (+1 or -1), in the
// scan precision; in MIXED, guarded like the scan's points.  Every lane of the
// warp computes the same value.
template <typename TS, typename TP>
__device__ __forceinline__ TS scan_point(const Solve<TS, TP>& v, int kernel, double h, int kk, int sgn) {
    const float hf = float(h), hl = float(h - double(hf));
    const TS x = grid_point(TS(kk), h, hf, hl);
    if constexpr (sizeof(TS) != sizeof(TP)) {
        bool need = false;
        const TS f = residual_guarded(v.ms, v.ss, v.cs, sgn < 0 ? -x : x, v.mode, kernel, need);
        if (!need) return f;
        return narrow_sign(residual_cold(v.mp, v.sp, v.cp, TP(double(sgn) * (double(kk) * h)), v.mode, kernel));
    } else {
        return residual(v.ms, v.ss, v.cs, sgn < 0 ? -x : x, v.mode, kernel);
    }
}

// Outward scan of the grid distances kk in [k_begin, k_end] on both sides by
// one warp.  fb_pos / fb_neg are the residuals at +-(k_begin-1)h.  Candidates
// are taken in order of |vartheta| (brackets at inner distance kk-1 before the
// exact zeros at kk; on one key the smaller polished |vartheta|, the negative
// root on a tie); returns true with the first decaying root.
template <typename TS, typename TP>
__device__ bool scan_window(const Solve<TS, TP>& v, int kernel, double h, int k_begin, int k_end,
                            TS fb_pos, TS fb_neg, int lane, TP& root, RayQ<TP>& fq) {
    constexpr bool mixed = sizeof(TS) != sizeof(TP);
    constexpr int P = 4;     // consecutive grid points per lane per step
    const int mode = v.mode;
    const float hf = float(h), hl = float(h - double(hf));
    TS prev_pos = fb_pos, prev_neg = fb_neg;
    for (int base = k_begin - 1; base < k_end; base += 16 * P) {
        const bool neg = lane >= 16;
        const int l16 = lane & 15;
        const int k0 = base + 1 + l16 * P;
        const TS kf0 = TS(k0);
        TS fv[P];
        if constexpr (mixed) {
            bool need[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const TS xk = grid_point(kf0 + TS(p), h, hf, hl);
                need[p] = false;
                fv[p] = k0 + p <= k_end ? residual_guarded(v.ms, v.ss, v.cs, neg ? -xk : xk, mode, kernel, need[p])
                                        : TS(NAN);
            }
            guard_points<TP>(v, kernel, h, base, fv, need, lane);
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const TS xk = grid_point(kf0 + TS(p), h, hf, hl);
                fv[p] = k0 + p <= k_end ? residual(v.ms, v.ss, v.cs, neg ? -xk : xk, mode, kernel) : TS(NAN);
            }
        }
        TS before = __shfl_up_sync(0xffffffffu, fv[P - 1], 1);    // point just inside
        if (l16 == 0) before = neg ? prev_neg : prev_pos;
        unsigned bm[P], zm[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const TS fprev = p == 0 ? before : fv[p - 1];
            // strict sign change (a product could underflow for the tiny
            // guarded values that narrow_sign returns)
            bm[p] = __ballot_sync(0xffffffffu, (fprev < TS(0) && fv[p] > TS(0)) || (fprev > TS(0) && fv[p] < TS(0)));
            zm[p] = __ballot_sync(0xffffffffu, fv[p] == TS(0));
        }
        prev_pos = __shfl_sync(0xffffffffu, fv[P - 1], 15);
        prev_neg = __shfl_sync(0xffffffffu, fv[P - 1], 31);
        unsigned anyb = 0, anyz = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) { anyb |= bm[p]; anyz |= zm[p]; }
        unsigned lanes = (anyb | anyz);
        lanes = (lanes | (lanes >> 16)) & 0xffffu;
        while (lanes) {
            const int l = __ffs(lanes) - 1;
            lanes &= lanes - 1;
            for (int p = 0; p < P; ++p) {
                const double kkl = static_cast<double>(base + 1 + l * P + p);
                TP cand[2];
                bool cok[2] = {false, false};
                RayQ<TP> cq[2];
                for (int side = 0; side < 2; ++side) {      // 0: negative, 1: positive
                    const int ln = side ? l : 16 + l;
                    if (!((bm[p] >> ln) & 1u)) continue;
                    const TS fcur = __shfl_sync(0xffffffffu, fv[p], ln);
                    const TS fin = __shfl_sync(0xffffffffu, p == 0 ? before : fv[p > 0 ? p - 1 : 0], ln);
                    const TS fl = side ? fin : fcur, fh = side ? fcur : fin;
                    const double glo = side ? (kkl - 1.0) * h : -kkl * h;
                    const double ghi = side ? kkl * h : -(kkl - 1.0) * h;
                    // polish in the scan precision (float for FP32 and MIXED); in
                    // MIXED it only seeds the refinement window of +-h/4, so
                    // h/64 is enough
                    const TS stop = sizeof(TS) == 8 ? TS(1e-9) : mixed ? TS(h / 64) : TS(0);
                    const TS rs = polish(v.ms, v.ss, v.cs, mode, kernel, TS(glo), TS(ghi), fl, fh, lane, stop);
                    if constexpr (mixed) {
                        // drop clearly growing roots in float; decide the rest in TP
                        const RayQ<TS> q32 = ray_quantities(v.ms, v.ss, v.cs, rs, mode, kernel);
                        if (!(q32.vi <= TS(1e-4) * q32.vr)) continue;
                        const Refined<TP> rf = refine<TP>(v.mp, v.sp, v.cp, mode, kernel, TP(rs), TP(glo), TP(ghi),
                                                          lane);
                        cq[side] = rf.q;
                        cand[side] = rf.root;
                    } else {
                        cq[side] = ray_quantities(v.mp, v.sp, v.cp, TP(rs), mode, kernel);
                        cand[side] = TP(rs);
                    }
                    cok[side] = cq[side].ok;
                }
                if (cok[0] || cok[1]) {
                    const int pick = (cok[0] && cok[1]) ? (fabs(cand[1]) < fabs(cand[0]) ? 1 : 0)
                                                        : (cok[0] ? 0 : 1);
                    root = cand[pick];
                    fq = cq[pick];
                    return true;
                }
                for (int side = 0; side < 2; ++side) {   // negative first
                    const int ln = side ? l : 16 + l;
                    if (!((zm[p] >> ln) & 1u)) continue;
                    const TP r = side ? TP(kkl * h) : TP(-kkl * h);
                    const RayQ<TP> q = ray_quantities(v.mp, v.sp, v.cp, r, mode, kernel);
                    if (q.ok) { root = r; fq = q; return true; }
                }
            }
        }
    }
    return false;
}

__device__ __forceinline__ size_t entry_index(int mi, int k, int n_classes, const Geo& g, int d) {
    return (static_cast<size_t>(mi) * n_classes + k) * g.n_dir() + d;
}

// Write the up to four mirrored entries of a folded solve (lanes 0..3), the
// ray direction reflected into the quadrant of theta_d, then rotated by the
// tilt (Eq. 36).
template <typename TS, typename TP, typename TO>
__device__ void write_entries(const Outs& out, const Solve<TS, TP>& v, int n_classes, const Geo& g,
                              bool found, TP root, const RayQ<TP>& q, int lane) {
    const int j = v.j;
    if (g.three_d()) {
        // one entry: the sagittal ray turned to the local azimuth, mirrored in
        // z' where the local polar angle was folded, expressed globally (Eq. 35)
        if (lane != 0) return;
        const size_t e = entry_index(v.mi, v.k, n_classes, g, j);
        double th, ph, n[3], E[3][3];
        global_direction(g, j, th, ph, n);
        put<TO>(out.theta, e, th);
        put<TO>(out.phi, e, ph);
        if (found) {
            local_basis(v.cls.tilt, v.cls.azim, E);
            double sp, cp;
            sincos(v.phl, &sp, &cp);
            const double rs = double(q.rx);
            const double rl[3] = {rs * cp, rs * sp, v.sz * double(q.rz)};
            double r[3];
            for (int c = 0; c < 3; ++c)
                r[c] = __fma_rn(E[2][c], rl[2], __fma_rn(E[1][c], rl[1], __dmul_rn(E[0][c], rl[0])));
            put<TO>(out.rx, e, r[0]);
            put<TO>(out.ry, e, r[1]);
            put<TO>(out.rz, e, r[2]);
            put<TO>(out.V, e, double(q.V));
            put<TO>(out.A, e, double(q.A));
            put<TO>(out.Q, e, double(q.Q));
            put<TO>(out.vartheta, e, double(root) * v.sz);
            out.flag[e] = 0;
        } else {
            put<TO>(out.rx, e, NAN);
            put<TO>(out.ry, e, NAN);
            put<TO>(out.rz, e, NAN);
            put<TO>(out.V, e, NAN);
            put<TO>(out.A, e, NAN);
            put<TO>(out.Q, e, NAN);
            put<TO>(out.vartheta, e, NAN);
            out.flag[e] = 1;
        }
        return;
    }
    const int M = g.M;
    int d, sx, sz, cnt;
    if (j == 0) {
        cnt = 2;
        d = lane == 0 ? 0 : 2 * M; sx = lane == 0 ? 1 : -1; sz = sx;
    } else if (j == M) {
        cnt = 2;
        d = lane == 0 ? M : 3 * M; sx = lane == 0 ? 1 : -1; sz = -sx;
    } else {
        cnt = 4;
        d = lane == 0 ? j : lane == 1 ? 2 * M - j : lane == 2 ? 2 * M + j : 4 * M - j;
        sx = lane < 2 ? 1 : -1;
        sz = (lane == 0 || lane == 3) ? 1 : -1;
    }
    if (lane >= cnt) return;
    const size_t e = entry_index(v.mi, v.k, n_classes, g, d);
    double ct, st;
    sincos(v.cls.tilt, &st, &ct);
    put<TO>(out.theta, e, (M_PI / 2 * d) / M + v.cls.tilt);
    if (found) {
        // the tilt rotation with its roundings spelled out, so that every
        // kernel that writes entries rounds it alike
        const double lx = sx * double(q.rx), lz = sz * double(q.rz);
        put<TO>(out.rx, e, __fma_rn(lx, ct, __dmul_rn(lz, st)));
        put<TO>(out.rz, e, __fma_rn(lz, ct, -__dmul_rn(lx, st)));
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

// First launch: one warp per solve scans the first kPhase1Reach grid points per
// side (the bulk of the roots lie there); solves that need a longer scan are
// left marked kPending for the second launch.
// TS: scan precision, TP: polish + ray-quantity precision, TO: storage.
// With a solve list (items != NULL) warp w takes solve items[w]; a solve is
// numbered mode_slot*n_classes*P + class*P + j with P = M+1 (2D) or
// n_az*n_pol (3D, j the entry d).
// With a device-side count (n_dev != NULL: the list length is known only on
// the device, e.g. inside a CUDA graph) the grid is sized for the machine and
// each warp strides over the list.
template <typename TS, typename TP, typename TO>
__device__ __forceinline__ void build_solve(const chert_class* __restrict__ classes, int n_classes,
                                            const ModeList& modes, const Geo& g, double h, int K, int kernel,
                                            const Outs& out, long long idx, int lane) {
    const Solve<TS, TP> v = make_solve<TS, TP>(classes, n_classes, modes, g, idx);
    bool found = false;
    TP root = TP(0);
    RayQ<TP> fq{};
    const TS f0 = scan_point(v, kernel, h, 0, 1);
    if (f0 == TS(0)) {
        const RayQ<TP> q = ray_quantities(v.mp, v.sp, v.cp, TP(0), v.mode, kernel);
        if (q.ok) { found = true; fq = q; }
    }
    const int reach = min(K, kPhase1Reach);
    if (!found) found = scan_window(v, kernel, h, 1, reach, f0, f0, lane, root, fq);
    if (!found && K > reach) {
        if (lane == 0) out.flag[entry_index(v.mi, v.k, n_classes, g, v.j)] = kPending;
        return;
    }
    write_entries<TS, TP, TO>(out, v, n_classes, g, found, root, fq, lane);
}

// DEV: the list length is *n_dev (a separate instantiation, so that the
// common form keeps its register allocation).
template <typename TS, typename TP, typename TO, bool DEV>
__global__ void __launch_bounds__(256, 2) cache_build_kernel(const chert_class* __restrict__ classes,
                                                          int n_classes, ModeList modes, Geo g,
                                                          double h, int K, int kernel, Outs out,
                                                          const int64_t* __restrict__ items,
                                                          long long n_items, const long long* __restrict__ n_dev) {
    const int lane = threadIdx.x & 31;
    const long long warp = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if constexpr (DEV) {
        const long long total = *n_dev;
        const long long stride = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
        for (long long w = warp; w < total; w += stride)
            build_solve<TS, TP, TO>(classes, n_classes, modes, g, h, K, kernel, out, items[w], lane);
    } else {
        const long long total = items ? n_items : static_cast<long long>(modes.n) * n_classes * g.per_class();
        if (warp >= total) return;
        build_solve<TS, TP, TO>(classes, n_classes, modes, g, h, K, kernel, out, items ? items[warp] : warp, lane);
    }
}

// Second launch: one 1024-thread CTA per chunk of `chunk` (<= kFinishChunk)
// consecutive solves (of the solve list, if any).  It collects the chunk's
// pending solves in shared memory and finishes them one after another with
// the whole CTA: each round its 32 warps scan consecutive 64-point slices of
// grid distance (2048 per side per round); the nearest slice with a decaying
// root wins.  The host sizes the chunks so that large builds launch few CTAs
// and small ones still spread their pending solves over every SM; the block
// scheduler balances the uneven work.
constexpr int kFinishChunk = 256;

template <typename TS, typename TP, typename TO, int NT>
__device__ void finish_one(const chert_class* __restrict__ classes, int n_classes, const ModeList& modes,
                           const Geo& g, double h, int K, int kernel, const Outs& out, long long idx) {
    constexpr int NW = NT / 32;
    __shared__ int s_found[NW];
    __shared__ double s_root[NW];
    __shared__ RayQ<TP> s_q[NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const Solve<TS, TP> v = make_solve<TS, TP>(classes, n_classes, modes, g, idx);
    constexpr int slice = 64;
    int winner = -1;
    for (int r0 = kPhase1Reach; r0 < K && winner < 0; r0 += NW * slice) {
        const int kb = r0 + w * slice + 1, ke = min(K, r0 + (w + 1) * slice);
        bool found = false;
        TP root = TP(0);
        RayQ<TP> q{};
        if (kb <= ke) {
            const TS fp = scan_point(v, kernel, h, kb - 1, 1);
            const TS fn = scan_point(v, kernel, h, kb - 1, -1);
            found = scan_window(v, kernel, h, kb, ke, fp, fn, lane, root, q);
        }
        if (lane == 0) {
            s_found[w] = found;
            s_root[w] = double(root);
            s_q[w] = q;
        }
        __syncthreads();
        for (int i = 0; i < NW; ++i)
            if (s_found[i]) { winner = i; break; }
        __syncthreads();
    }
    if (w == 0) {
        const bool found = winner >= 0;
        const TP root = found ? TP(s_root[winner]) : TP(0);
        const RayQ<TP> q = found ? s_q[winner] : RayQ<TP>{};
        write_entries<TS, TP, TO>(out, v, n_classes, g, found, root, q, lane);
    }
    __syncthreads();
}

template <typename TS, typename TP, typename TO, int NT>
__device__ __forceinline__ void finish_chunk(const chert_class* __restrict__ classes, int n_classes,
                                             const ModeList& modes, const Geo& g, double h, int K, int kernel,
                                             const Outs& out, const int64_t* __restrict__ items, long long n_total,
                                             int chunk, long long base, long long* s_list, int* s_count) {
    const int per = g.per_class();
    if (threadIdx.x == 0) *s_count = 0;
    __syncthreads();
    const long long t = base + threadIdx.x;
    if ((int)threadIdx.x < chunk && t < n_total) {
        const long long idx = items ? items[t] : t;
        const int j = static_cast<int>(idx % per);
        const int k = static_cast<int>((idx / per) % n_classes);
        const int mi = static_cast<int>(idx / (static_cast<long long>(per) * n_classes));
        if (out.flag[entry_index(mi, k, n_classes, g, j)] == kPending) s_list[atomicAdd(s_count, 1)] = idx;
    }
    __syncthreads();
    const int cnt = *s_count;
    for (int q = 0; q < cnt; ++q)
        finish_one<TS, TP, TO, NT>(classes, n_classes, modes, g, h, K, kernel, out, s_list[q]);
}

// DEV: the list length is *n_dev and the CTAs stride over the chunks.
// NT threads per CTA: 1024 (64 registers a thread) finishes a solve's scan
// in the fewest rounds; 256 (128 registers, two CTAs an SM) spills less.
template <typename TS, typename TP, typename TO, bool DEV, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) cache_finish_kernel(const chert_class* __restrict__ classes,
                                                            int n_classes, ModeList modes, Geo g,
                                                            double h, int K, int kernel, Outs out,
                                                            const int64_t* __restrict__ items,
                                                            long long n_total, int chunk,
                                                            const long long* __restrict__ n_dev) {
    __shared__ long long s_list[kFinishChunk];
    __shared__ int s_count;
    if constexpr (DEV) {
        const long long n = *n_dev;
        for (long long base = (long long)blockIdx.x * chunk; base < n; base += (long long)gridDim.x * chunk) {
            finish_chunk<TS, TP, TO, NT>(classes, n_classes, modes, g, h, K, kernel, out, items, n, chunk, base,
                                         s_list, &s_count);
            __syncthreads();
        }
    } else {
        finish_chunk<TS, TP, TO, NT>(classes, n_classes, modes, g, h, K, kernel, out, items, n_total, chunk,
                                     (long long)blockIdx.x * chunk, s_list, &s_count);
    }
}

}  // namespace
}  // namespace chert

// d_n_items != NULL: the solve list d_items holds *d_n_items entries (a count
// on the device, at most n_items); the launches are sized for the machine and
// stride over the list, so no host read of the count is needed.
std::atomic<int> g_finish_threads{0};     // 0: the default

static int launch_build(const chert_class* d_classes, int n_classes, const int* modes, int n_modes,
                        const chert_cache_params* params, const chert_cache_arrays* out,
                        const int64_t* d_items, long long n_items, void* stream, const char* who,
                        int n_az = 0, int n_pol = 0, const long long* d_n_items = nullptr) {
    using namespace chert;
    CHERT_REQUIRE(d_classes && modes && params && out, "%s: NULL argument", who);
    CHERT_REQUIRE(n_classes >= 1, "%s: n_classes=%d", who, n_classes);
    CHERT_REQUIRE(n_modes >= 1 && n_modes <= 3, "%s: n_modes=%d", who, n_modes);
    CHERT_REQUIRE(n_az > 0 || (params->M >= 1 && params->M <= (1 << 20)), "%s: M=%d", who, params->M);
    CHERT_REQUIRE(n_az == 0 || (n_az >= 1 && n_pol >= 1 && (long long)n_az * n_pol <= (1 << 24)),
                  "%s: n_az=%d n_pol=%d", who, n_az, n_pol);
    CHERT_REQUIRE(n_az == 0 || out->ry, "%s: a 3D cache needs the ry output", who);
    CHERT_REQUIRE(params->scan_step > 0 && params->scan_half >= 1 && params->scan_half <= (1 << 28),
                  "%s: bad scan grid", who);
    CHERT_REQUIRE(params->kernel == CHERT_OEV || params->kernel == CHERT_MEV, "%s: kernel=%d", who,
                  params->kernel);
    CHERT_REQUIRE(out->V && out->rx && out->rz && out->flag, "%s: V, rx, rz and flag outputs are required", who);
    ModeList ml{{0, 0, 0}, n_modes};
    for (int i = 0; i < n_modes; i++) {
        CHERT_REQUIRE(modes[i] >= CHERT_QP && modes[i] <= CHERT_QSH, "%s: mode %d", who, modes[i]);
        for (int j = 0; j < i; j++) CHERT_REQUIRE(modes[j] != modes[i], "%s: repeated mode", who);
        ml.m[i] = modes[i];
    }
    Outs o{out->V, out->A, out->Q, out->rx, out->rz, out->theta, out->vartheta, out->flag, out->ry, out->phi};
    const Geo geo{params->M, n_az, n_pol};
    const long long warps = d_items ? n_items : static_cast<long long>(n_modes) * n_classes * geo.per_class();
    if (warps == 0) return CHERT_OK;
    const int threads = 256;
    const long long blocks = (warps * 32 + threads - 1) / threads;
    CHERT_REQUIRE(blocks < (1LL << 31), "%s: problem too large", who);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double h = params->scan_step;
    const int K = params->scan_half;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) {
        cudaGetLastError();
        n_sm = 148;
    }
    const long long per_cta = (warps + 8LL * n_sm - 1) / (8LL * n_sm);        // ~8 CTAs per SM
    const int chunk = (int)std::max(1LL, std::min<long long>(kFinishChunk, per_cta));
    unsigned finish_blocks = (unsigned)((warps + chunk - 1) / chunk);
    unsigned build_blocks = (unsigned)blocks;
    if (d_n_items) {          // strided launches: 2 CTAs per SM of each kernel (its occupancy)
        build_blocks = (unsigned)std::min<long long>(blocks, 2LL * n_sm);
        finish_blocks = (unsigned)std::min<long long>(finish_blocks, 2LL * n_sm);
    }
    const int kern = params->kernel;
    // finish pass: 1024 threads a CTA for small builds (the fewest rounds per
    // pending solve: latency), 256 for large ones (no register cap of 64, so
    // fewer spills: throughput; 15% faster on a 10.9M-solve build)
    const int finish_nt = g_finish_threads.load() ? g_finish_threads.load() : (warps <= (1LL << 16) ? 1024 : 256);
#define CHERT_LAUNCH_BUILD_DEV(TS, TP, TO, DEV)                                                         \
    cache_build_kernel<TS, TP, TO, DEV><<<build_blocks, threads, 0, s>>>(d_classes, n_classes, ml, geo, h, K, \
                                                                        kern, o, d_items, n_items, d_n_items); \
    if (K > kPhase1Reach)                                                                               \
        switch (finish_nt) {                                                                            \
            case 256: cache_finish_kernel<TS, TP, TO, DEV, 256><<<finish_blocks, 256, 0, s>>>(              \
                          d_classes, n_classes, ml, geo, h, K, kern, o, d_items, warps, chunk, d_n_items); break; \
            case 512: cache_finish_kernel<TS, TP, TO, DEV, 512><<<finish_blocks, 512, 0, s>>>(              \
                          d_classes, n_classes, ml, geo, h, K, kern, o, d_items, warps, chunk, d_n_items); break; \
            default: cache_finish_kernel<TS, TP, TO, DEV, 1024><<<finish_blocks, 1024, 0, s>>>(             \
                          d_classes, n_classes, ml, geo, h, K, kern, o, d_items, warps, chunk, d_n_items);       \
        }
#define CHERT_LAUNCH_BUILD(TS, TP, TO)                                                                  \
    if (d_n_items) { CHERT_LAUNCH_BUILD_DEV(TS, TP, TO, true) } else { CHERT_LAUNCH_BUILD_DEV(TS, TP, TO, false) }
    switch (params->precision) {
        case CHERT_FP64: CHERT_LAUNCH_BUILD(double, double, double) break;
        case CHERT_FP32: CHERT_LAUNCH_BUILD(float, float, float) break;
        case CHERT_MIXED: CHERT_LAUNCH_BUILD(float, xf::ff, float) break;
        default: CHERT_REQUIRE(false, "%s: precision=%d", who, params->precision);
    }
#undef CHERT_LAUNCH_BUILD
#undef CHERT_LAUNCH_BUILD_DEV
    return launch_check(who);
}

extern "C" int chert_build_cache(const chert_class* d_classes, int n_classes, const int* modes,
                                 int n_modes, const chert_cache_params* params,
                                 const chert_cache_arrays* out, void* stream) {
    return launch_build(d_classes, n_classes, modes, n_modes, params, out, nullptr, 0, stream,
                        "chert_build_cache");
}

extern "C" int chert_build_cache_items(const chert_class* d_classes, int n_classes, const int* modes,
                                       int n_modes, const chert_cache_params* params,
                                       const int64_t* d_items, int64_t n_items,
                                       const chert_cache_arrays* out, void* stream) {
    CHERT_REQUIRE(d_items && n_items >= 0, "chert_build_cache_items: bad item list");
    return launch_build(d_classes, n_classes, modes, n_modes, params, out, d_items, n_items, stream,
                        "chert_build_cache_items");
}

namespace chert {
int surrogate_cache(const float* const* d_params_per_mode, const chert_class* d_classes, int n_classes,
                    const int* modes, int n_modes, int M, int precision, const chert_cache_arrays* out,
                    void* d_ws, size_t ws_bytes, void* stream, bool check);
}

// The solves a surrogate cache hands to the exact solver (flag 2 on the
// solve's own entry, d = j): compacted into a list with a device-side count.
__global__ void collect_fallback_kernel(const uint8_t* __restrict__ flag, int n_modes, int n_classes, int M,
                                        int64_t* __restrict__ items, unsigned long long* __restrict__ count) {
    const long long per = M + 1;
    const long long n = (long long)n_modes * n_classes * per;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool take = false;
    if (t < n) {
        const long long j = t % per, mk = t / per;             // mk = mode slot * n_classes + class
        take = flag[mk * 4 * M + j] == 2;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, take);
    unsigned long long base = 0;
    const int lane = threadIdx.x & 31;
    if (lane == 0 && ballot) base = atomicAdd(count, (unsigned long long)__popc(ballot));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (take) items[base + __popc(ballot & ((1u << lane) - 1))] = t;
}

extern "C" size_t chert_cache_surrogate_workspace_bytes(int n_classes, int n_modes, int M) {
    if (n_classes < 1 || n_modes < 1 || n_modes > 3 || M < 1) return 0;
    const size_t s = chert_surrogate_cache_workspace_bytes(n_classes, M);
    if (s == 0) return 0;
    auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
    return a256(s) + a256(8 * (size_t)n_modes * n_classes * (M + 1)) + 256;
}

extern "C" int chert_cache_surrogate(const float* const* d_params_per_mode, const chert_class* d_classes,
                                     int n_classes, const int* modes, int n_modes,
                                     const chert_cache_params* params, const chert_cache_arrays* out,
                                     void* d_ws, size_t ws_bytes, int64_t* d_n_fallback, void* stream) {
    using namespace chert;
    const char* who = "chert_cache_surrogate";
    CHERT_REQUIRE(d_params_per_mode && d_classes && modes && params && out && d_ws, "%s: NULL argument", who);
    const size_t need = chert_cache_surrogate_workspace_bytes(n_classes, n_modes, params->M);
    CHERT_REQUIRE(need > 0, "%s: n_classes=%d n_modes=%d M=%d", who, n_classes, n_modes, params->M);
    if (ws_bytes < need) {
        set_error("%s: workspace %zu < %zu bytes", who, ws_bytes, need);
        return CHERT_ENOMEM;
    }
    auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t s_bytes = chert_surrogate_cache_workspace_bytes(n_classes, params->M);
    unsigned char* w = static_cast<unsigned char*>(d_ws);
    int64_t* items = reinterpret_cast<int64_t*>(w + a256(s_bytes));
    unsigned long long* count =
        reinterpret_cast<unsigned long long*>(w + a256(s_bytes) + a256(8 * (size_t)n_modes * n_classes * (params->M + 1)));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int net_prec = params->precision == CHERT_FP64 ? CHERT_FP64 : CHERT_FP32;
    int rc = surrogate_cache(d_params_per_mode, d_classes, n_classes, modes, n_modes, params->M, net_prec, out, d_ws,
                             s_bytes, stream, false);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(*count), s);
    if (e != cudaSuccess) return cuda_fail(e, "chert_cache_surrogate: count reset");
    const long long n = (long long)n_modes * n_classes * (params->M + 1);
    collect_fallback_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out->flag, n_modes, n_classes, params->M,
                                                                         items, count);
    rc = launch_check("chert_cache_surrogate: fallback list");
    if (rc) return rc;
    rc = launch_build(d_classes, n_classes, modes, n_modes, params, out, items, n, stream, who, 0, 0,
                      reinterpret_cast<const long long*>(count));
    if (rc) return rc;
    if (d_n_fallback) {
        e = cudaMemcpyAsync(d_n_fallback, count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "chert_cache_surrogate: count copy");
    }
    return CHERT_OK;
}

extern "C" int chert_build_cache_3d(const chert_class* d_classes, int n_classes, const int* modes, int n_modes,
                                    int n_az, int n_pol, const chert_cache_params* params,
                                    const chert_cache_arrays* out, void* stream) {
    CHERT_REQUIRE(n_az >= 1 && n_pol >= 1, "chert_build_cache_3d: n_az=%d n_pol=%d", n_az, n_pol);
    return launch_build(d_classes, n_classes, modes, n_modes, params, out, nullptr, 0, stream,
                        "chert_build_cache_3d", n_az, n_pol);
}

extern "C" int chert_set_cache_finish_threads(int threads) {
    CHERT_REQUIRE(threads == 0 || threads == 256 || threads == 512 || threads == 1024,
                  "chert_set_cache_finish_threads: threads=%d (0, 256, 512 or 1024)", threads);
    return g_finish_threads.exchange(threads);
}

extern "C" int chert_cache_eval_counter(int enable, unsigned long long* counts_out) {
    using namespace chert;
    cudaError_t e;
    if (enable) {
        const unsigned long long zero[3] = {0, 0, 0};
        const int on = 1;
        e = cudaMemcpyToSymbol(g_eval_count, zero, sizeof(zero));
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_eval_count_on, &on, sizeof(on));
        if (e != cudaSuccess) return cuda_fail(e, "chert_cache_eval_counter: enable");
        return CHERT_OK;
    }
    const int off = 0;
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_eval_count_on, &off, sizeof(off));
    unsigned long long c[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(c, g_eval_count, sizeof(c));
    if (e != cudaSuccess) return cuda_fail(e, "chert_cache_eval_counter: read");
    if (counts_out)
        for (int i = 0; i < 3; ++i) counts_out[i] = c[i];
    return CHERT_OK;
}
