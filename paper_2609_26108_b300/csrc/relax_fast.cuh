// Relaxation specialised to the standard secondary-node stencil: all lattice
// directions (ox, oz) with max(|ox|, |oz|) <= R and gcd(|ox|, |oz|) = 1.
//
// Same algorithm and results as the generic relax_kernel (sweep cycles, then a
// verification pass that yields the parents), but the stencil is a
// compile-time table, so every pull compiles to
//   LDS tau_i [lag-row base - ox] ; LDS k_i [class-row base - ox] ;
//   IADD ; LDS w [W_j + k_i + o] ; FADD ; FMNMX
// with immediate offsets:
//   * lines live in a ring of 8 (sweeps) or 16 (verification) shared-memory
//     rows padded by R on both sides with +inf, so no pull needs a bounds test;
//   * class ids are stored pre-multiplied (k * nk * n_off) so that the weight
//     table W[k_i][k_j][o] is addressed by one add;
//   * the next line's tau and class are loaded from global memory while the
//     current line is pulled.
// The verification pass pulls each node's in-neighbours in increasing node
// index, so a strict '<' keeps the smallest index on ties (the parent rule).
#pragma once
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace chert {
namespace fast {

constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }
constexpr int cabs(int a) { return a < 0 ? -a : a; }

template <int R>
constexpr int stencil_count() {
    int n = 0;
    for (int z = -R; z <= R; ++z)
        for (int x = -R; x <= R; ++x)
            if ((x || z) && cgcd(cabs(x), cabs(z)) == 1) ++n;
    return n;
}

template <int R>
struct Stencil {
    static constexpr int N = stencil_count<R>();
    int x[N], z[N];
    // order: oz descending, then ox descending -> increasing i = j - o
    constexpr Stencil() : x(), z() {
        int n = 0;
        for (int zz = R; zz >= -R; --zz)
            for (int xx = R; xx >= -R; --xx)
                if ((xx || zz) && cgcd(cabs(xx), cabs(zz)) == 1) {
                    x[n] = xx;
                    z[n] = zz;
                    ++n;
                }
    }
};

// The table as a constant expression usable inside device code.
template <int R>
struct Table {
    static constexpr Stencil<R> v{};
};

// Compile-time loop: f(std::integral_constant<int, Q>) for Q = 0 .. N-1.
template <typename F, int... Q>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Q...>) {
    (f(std::integral_constant<int, Q>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

}  // namespace fast
}  // namespace chert

namespace chert {
namespace fast {

// Per-launch arguments of the specialised kernel (FieldArgs of the generic one
// plus the map from stencil index to the caller's offset index).
struct Args {
    int nx, nz, n_classes, n_modes, max_cycles;
    double dx;
    const int32_t* cls;
    const int64_t* src;
    void *tauR, *tauI;
    int32_t *parR, *parI;
    const void *Vsel, *Asel;   // [n_modes][n_classes][n_off] in the caller's offset order
    int n_off;
    int* status;
    short map[128];            // stencil index -> caller offset index
};

// One ring element: the node's tau and its class id pre-multiplied by nk*N,
// read by a single 8-byte (float) or 16-byte (double) shared load.
template <typename T>
struct alignas(2 * sizeof(T)) Cell {
    T tau;
    int ck;
};

template <typename T>
struct Ctx {
    T* W;            // [nk][nk][N]: W[(ki*nk + kj)*N + q]
    Cell<T>* ring;   // [16][LS]
    short* sx;       // stencil offsets (for decoding the winning parent)
    short* sz;
    int LS, nx, nz, nk;
};

__device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double fmin_(double a, double b) { return fmin(a, b); }

// One sweep over lines along AXIS (0: rows in z, 1: columns in x) in
// direction DIR; every node pulls from its in-neighbours on the previous
// lines (offsets whose across-line component has the sign of DIR).
template <typename T, int R, int PPT, int AXIS, int DIR>
__device__ void sweep(const Ctx<T>& c, T* __restrict__ tau, const int32_t* __restrict__ cls) {
    constexpr int N = Stencil<R>::N;
    const int n_lines = AXIS == 0 ? c.nz : c.nx;
    const int len = AXIS == 0 ? c.nx : c.nz;
    const int nx = c.nx;
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int i = tid; i < 8 * c.LS; i += bd) c.ring[i] = Cell<T>{T(INFINITY), 0};
    __syncthreads();
    T cur[PPT];
    int kr[PPT];
    auto load = [&](int line, T* t, int* k) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int u = tid + p * bd;
            if (u < len) {
                const size_t j = AXIS == 0 ? (size_t)u + (size_t)nx * line : (size_t)line + (size_t)nx * u;
                t[p] = tau[j];
                k[p] = min(max(cls[j], 0), c.nk - 1);
            }
        }
    };
    load(DIR > 0 ? 0 : n_lines - 1, cur, kr);
    for (int step = 0; step < n_lines; ++step) {
        const int line = DIR > 0 ? step : n_lines - 1 - step;
        T nxt[PPT];
        int nkr[PPT];
        if (step + 1 < n_lines) load(DIR > 0 ? line + 1 : line - 1, nxt, nkr);
        const Cell<T>* pt[R + 1];
#pragma unroll
        for (int lag = 1; lag <= R; ++lag) pt[lag] = c.ring + ((line - DIR * lag) & 7) * c.LS + R;
        const int own = (line & 7) * c.LS + R;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int u = tid + p * bd;
            if (u < len) {
                const T* Wj = c.W + kr[p] * N;
                T best = cur[p];
                static_for<N>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    constexpr int oa = AXIS == 0 ? Table<R>::v.z[q] : Table<R>::v.x[q];
                    constexpr int ol = AXIS == 0 ? Table<R>::v.x[q] : Table<R>::v.z[q];
                    if constexpr (oa * DIR > 0) {
                        constexpr int lag = oa * DIR;
                        const Cell<T> ci = pt[lag][u - ol];
                        best = fmin_(best, ci.tau + Wj[ci.ck + q]);
                    }
                });
                c.ring[own + u] = Cell<T>{best, kr[p] * c.nk * N};
                if (best < cur[p]) {
                    const size_t j = AXIS == 0 ? (size_t)u + (size_t)nx * line : (size_t)line + (size_t)nx * u;
                    tau[j] = best;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < PPT; ++p) { cur[p] = nxt[p]; kr[p] = nkr[p]; }
    }
}

// Verification pass over rows with a 16-row ring: pulls every in-neighbour in
// increasing node index; lowers tau where possible (returns whether anything
// changed) and otherwise writes the argmin parent.
template <typename T, int R, int PPT>
__device__ bool verify(const Ctx<T>& c, T* __restrict__ tau, const int32_t* __restrict__ cls,
                       int64_t src, int32_t* __restrict__ par) {
    constexpr int N = Stencil<R>::N;
    const int nx = c.nx, nz = c.nz;
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int i = tid; i < 16 * c.LS; i += bd) c.ring[i] = Cell<T>{T(INFINITY), 0};
    __syncthreads();
    auto store_row = [&](int row) {          // global row -> ring (inf beyond the lattice)
        const int base = (row & 15) * c.LS + R;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int x = tid + p * bd;
            if (x < nx) {
                if (row < nz) {
                    const size_t j = (size_t)x + (size_t)nx * row;
                    c.ring[base + x] = Cell<T>{tau[j], min(max(cls[j], 0), c.nk - 1) * c.nk * N};
                } else {
                    c.ring[base + x] = Cell<T>{T(INFINITY), 0};
                }
            }
        }
    };
    for (int row = 0; row < R && row < nz; ++row) store_row(row);
    bool changed = false;
    for (int z = 0; z < nz; ++z) {
        store_row(z + R);
        __syncthreads();
        const Cell<T>* pt[2 * R + 1];
#pragma unroll
        for (int d = -R; d <= R; ++d) pt[d + R] = c.ring + ((z - d) & 15) * c.LS + R;   // row z - d
        const int own = (z & 15) * c.LS + R;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int x = tid + p * bd;
            if (x < nx) {
                const Cell<T> me = c.ring[own + x];
                const T cur = me.tau;
                const int kj = me.ck / (c.nk * N);
                const T* Wj = c.W + kj * N;
                T best = T(INFINITY);
                int bq = -1;
                static_for<N>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    constexpr int oz = Table<R>::v.z[q], ox = Table<R>::v.x[q];
                    const Cell<T> ci = pt[oz + R][x - ox];
                    const T cand = ci.tau + Wj[ci.ck + q];
                    if (cand < best) { best = cand; bq = q; }
                });
                const size_t j = (size_t)x + (size_t)nx * z;
                if (best < cur) {
                    tau[j] = best;
                    changed = true;
                } else if (par) {
                    int32_t pj;
                    if ((int64_t)j == src) pj = (int32_t)src;
                    else if (isinf(cur) || bq < 0) pj = -1;
                    else pj = (int32_t)((long long)j - ((long long)c.sz[bq] * nx + c.sx[bq]));
                    par[j] = pj;
                }
            }
        }
    }
    return __syncthreads_or(changed);
}

template <typename T, int R, int PPT>
__global__ void __launch_bounds__(512) relax_fast_kernel(Args a) {
    constexpr int N = Stencil<R>::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = a.n_classes;
    const int field = blockIdx.x >> 1;
    const int comp = blockIdx.x & 1;
    const int mode = field % a.n_modes;
    const int s = field / a.n_modes;
    const int line_max = max(a.nx, a.nz);
    Ctx<T> c;
    c.nx = a.nx; c.nz = a.nz; c.nk = nk;
    c.LS = ((line_max + 2 * R) + 3) & ~3;
    unsigned char* p = smem_raw;
    c.W = reinterpret_cast<T*>(p); p += (size_t)nk * nk * N * sizeof(T);
    c.ring = reinterpret_cast<Cell<T>*>(p); p += (size_t)16 * c.LS * sizeof(Cell<T>);
    c.sx = reinterpret_cast<short*>(p); p += N * sizeof(short);
    c.sz = reinterpret_cast<short*>(p);

    const T* sel = static_cast<const T*>(comp == 0 ? a.Vsel : a.Asel) + (size_t)mode * nk * a.n_off;
    if (threadIdx.x == 0)
        static_for<N>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr short vx = Table<R>::v.x[q], vz = Table<R>::v.z[q];
            c.sx[q] = vx;
            c.sz[q] = vz;
        });
    __syncthreads();
    for (int t = threadIdx.x; t < nk * nk * N; t += blockDim.x) {
        const int q = t % N, kj = (t / N) % nk, ki = t / (N * nk);
        const int o = a.map[q];
        const double ox = c.sx[q], oz = c.sz[q];
        const T L = T(a.dx * sqrt(ox * ox + oz * oz));
        const T vi = sel[ki * a.n_off + o], vj = sel[kj * a.n_off + o];
        // Eq. 29-30 with the segment averages of Eq. 28 (same rounding as the
        // generic kernel: no contraction)
        c.W[t] = comp == 0 ? L / (T(0.5) * (vi + vj)) : L * (T(0.5) * (vi + vj));
    }

    const size_t n = (size_t)a.nx * a.nz;
    T* tau = static_cast<T*>(comp == 0 ? a.tauR : a.tauI) + (size_t)field * n;
    int32_t* par = comp == 0 ? a.parR : a.parI;
    if (par) par += (size_t)field * n;
    const int64_t src = a.src[s];
    for (size_t j = threadIdx.x; j < n; j += blockDim.x) tau[j] = (j == (size_t)src) ? T(0) : T(INFINITY);
    __syncthreads();

    int used = -1;
    for (int cycle = 0; cycle < a.max_cycles; ++cycle) {
        sweep<T, R, PPT, 0, +1>(c, tau, a.cls);
        sweep<T, R, PPT, 1, +1>(c, tau, a.cls);
        sweep<T, R, PPT, 1, -1>(c, tau, a.cls);
        sweep<T, R, PPT, 0, -1>(c, tau, a.cls);
        if (!verify<T, R, PPT>(c, tau, a.cls, src, par)) {
            used = cycle + 1;
            break;
        }
    }
    if (threadIdx.x == 0) a.status[blockIdx.x] = used;
}

}  // namespace fast
}  // namespace chert
