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
    // Per-node weights (used when the class-pair table does not fit in shared
    // memory): [n_modes*2 + comp][N][node], node index z*nx + x (row layout)
    // and x*nz + z (column layout); null for the class-pair table.
    const void *wrow, *wcol;
    // Row classes [nz]: rowk[z] = the class of every node of row z, or -1 if
    // the row holds several classes (written by row_classes_kernel); null
    // when the launch cannot use the row-class path.
    const int* rowk;
};

// One ring element: the node's tau and its class id pre-multiplied by nk*N,
// read by a single 8-byte (float) or 16-byte (double) shared load.
template <typename T>
struct alignas(2 * sizeof(T)) Cell {
    T tau;
    int ck;
};

// Dirty tiles.  The lattice is cut into kTile x kTile tiles; stamp[t] is the
// number of the last pass (counted over the whole run, from 1) in which a node
// of tile t was lowered.  A pull only reads nodes within R < kTile of the
// puller, i.e. in the 3 x 3 tiles around it, so a node whose surrounding tiles
// have not changed since the last pass of the same kind (sweep direction or
// verification) cannot improve, and its pulls are skipped.  The skip is exact:
// the results are those of the full passes.
constexpr int kTile = 32;

template <typename T>
struct Ctx {
    const int* rowk; // [nz] class of each row (row-class path), shared memory
    const int* rowoff; // rowoff[z] = rowk[z] * nk * N for z in [0, nz), 0 for the R rows
                       // either side (their traveltimes are +inf in the ring)
    T* W;            // [nk][nk][N]: W[(ki*nk + kj)*N + q] (class-pair mode)
    Cell<T>* ring;   // [16][LS]
    short* sx;       // stencil offsets (for decoding the winning parent)
    short* sz;
    int* stamp;      // [TZ][TX]
    const T* wr;     // per-node weights of this (mode, component), row layout
    const T* wc;     // column layout
    size_t n;        // nodes
    int LS, nx, nz, nk, TX, TZ;
};

__device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double fmin_(double a, double b) { return fmin(a, b); }

// Whether the tiles around tile (tx, tz) changed in or after pass `since`.
template <typename T>
__device__ __forceinline__ bool dirty(const Ctx<T>& c, int tx, int tz, int since) {
    if (since <= 0) return true;       // every stamp is >= 0: the first pass of a sweep relaxes everything
    int m = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int z = tz + dz;
        if (z < 0 || z >= c.TZ) continue;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int x = tx + dx;
            if (x < 0 || x >= c.TX) continue;
            m = max(m, c.stamp[z * c.TX + x]);
        }
    }
    return m >= since;
}

// Whether any tile of bands b-1..b+1 changed in or after pass `since`; a band
// is kTile consecutive lines across AXIS (0: rows, tile row b; 1: columns,
// tile column b).  Block-wide (every thread must call it).
template <typename T, int AXIS>
__device__ __forceinline__ bool band_dirty(const Ctx<T>& c, int b, int since) {
    if (since <= 0) return true;                // uniform over the block, as the barrier below
    const int nb = AXIS == 0 ? c.TZ : c.TX;     // bands
    const int per = AXIS == 0 ? c.TX : c.TZ;    // tiles per band
    bool d = false;
    for (int t = threadIdx.x; t < 3 * per; t += blockDim.x) {
        const int k = b - 1 + t / per, o = t % per;
        if (k < 0 || k >= nb) continue;
        const int tile = AXIS == 0 ? k * c.TX + o : o * c.TX + k;
        if (c.stamp[tile] >= since) d = true;
    }
    return __syncthreads_or(d);
}

// One sweep over lines along AXIS (0: rows in z, 1: columns in x) in
// direction DIR; every node pulls from its in-neighbours on the previous
// lines (offsets whose across-line component has the sign of DIR).  Pass
// number `pass`; `since` is the number of the previous pass of this sweep.
template <typename T, int R, int PPT, int AXIS, int DIR, bool PN>
__device__ void sweep(const Ctx<T>& c, T* __restrict__ tau, const int32_t* __restrict__ cls, int pass,
                      int since) {
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
                k[p] = PN ? 0 : min(max(cls[j], 0), c.nk - 1);
            }
        }
    };
    // Bands whose tiles and neighbouring tiles are all clean are skipped
    // whole (no node of them can change in this pass); the ring lines that the
    // next processed line reads are then reloaded from tau.
    auto ring_line = [&](int line) {
        Cell<T>* row = c.ring + (line & 7) * c.LS + R;
        const bool in = line >= 0 && line < n_lines;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int u = tid + p * bd;
            if (u < len) {
                if (in) {
                    const size_t j = AXIS == 0 ? (size_t)u + (size_t)nx * line : (size_t)line + (size_t)nx * u;
                    row[u] = Cell<T>{tau[j], PN ? 0 : min(max(cls[j], 0), c.nk - 1) * c.nk * N};
                } else {
                    row[u] = Cell<T>{T(INFINITY), 0};
                }
            }
        }
    };
    bool reload = false;
    load(DIR > 0 ? 0 : n_lines - 1, cur, kr);
    for (int step = 0; step < n_lines; ++step) {
        const int line = DIR > 0 ? step : n_lines - 1 - step;
        const bool band_start = DIR > 0 ? (line % kTile == 0) : (line == n_lines - 1 || line % kTile == kTile - 1);
        if (band_start) {
            const int b = line / kTile;
            if (!band_dirty<T, AXIS>(c, b, since)) {
                const int last = DIR > 0 ? min(n_lines - 1, b * kTile + kTile - 1) : b * kTile;
                step = DIR > 0 ? last : n_lines - 1 - last;      // the loop's ++step moves past it
                reload = true;
                continue;
            }
            if (reload) {
                for (int lag = 1; lag <= R; ++lag) ring_line(line - DIR * lag);
                load(line, cur, kr);
                __syncthreads();
                reload = false;
            }
        }
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
                const int tx = (AXIS == 0 ? u : line) / kTile, tz = (AXIS == 0 ? line : u) / kTile;
                T best = cur[p];
                if (dirty(c, tx, tz, since)) {          // uniform across the warp (one tile)
                    if constexpr (PN) {
                        const T* wl = (AXIS == 0 ? c.wr : c.wc) + (size_t)line * len + u;
                        static_for<N>([&](auto qc) {
                            constexpr int q = decltype(qc)::value;
                            constexpr int oa = AXIS == 0 ? Table<R>::v.z[q] : Table<R>::v.x[q];
                            constexpr int ol = AXIS == 0 ? Table<R>::v.x[q] : Table<R>::v.z[q];
                            if constexpr (oa * DIR > 0) {
                                constexpr int lag = oa * DIR;
                                best = fmin_(best, pt[lag][u - ol].tau + wl[(size_t)q * c.n]);
                            }
                        });
                    } else {
                        const T* Wj = c.W + kr[p] * N;
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
                    }
                }
                c.ring[own + u] = Cell<T>{best, kr[p] * c.nk * N};
                if (best < cur[p]) {
                    const size_t j = AXIS == 0 ? (size_t)u + (size_t)nx * line : (size_t)line + (size_t)nx * u;
                    tau[j] = best;
                    c.stamp[tz * c.TX + tx] = pass;
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
// changed) and otherwise writes the argmin parent.  Nodes of clean tiles keep
// the parent written when they were last verified: none of their
// in-neighbours has changed since.
template <typename T, int R, int PPT, bool PN>
__device__ bool verify(const Ctx<T>& c, T* __restrict__ tau, const int32_t* __restrict__ cls,
                       int64_t src, int32_t* __restrict__ par, int pass, int since) {
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
                if (row >= 0 && row < nz) {
                    const size_t j = (size_t)x + (size_t)nx * row;
                    c.ring[base + x] = Cell<T>{tau[j], PN ? 0 : min(max(cls[j], 0), c.nk - 1) * c.nk * N};
                } else {
                    c.ring[base + x] = Cell<T>{T(INFINITY), 0};
                }
            }
        }
    };
    for (int row = 0; row < R && row < nz; ++row) store_row(row);
    bool changed = false;
    bool reload = false;
    for (int z = 0; z < nz; ++z) {
        if (z % kTile == 0) {                     // skip clean bands of rows whole
            const int b = z / kTile;
            if (!band_dirty<T, 0>(c, b, since)) {
                z = min(nz, z + kTile) - 1;
                reload = true;
                continue;
            }
            if (reload) {
                for (int row = z - R; row < z + R; ++row) store_row(row);
                reload = false;
            }
        }
        store_row(z + R);
        __syncthreads();
        const Cell<T>* pt[2 * R + 1];
#pragma unroll
        for (int d = -R; d <= R; ++d) pt[d + R] = c.ring + ((z - d) & 15) * c.LS + R;   // row z - d
        const int own = (z & 15) * c.LS + R;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int x = tid + p * bd;
            if (x < nx && dirty(c, x / kTile, z / kTile, since)) {
                const Cell<T> me = c.ring[own + x];
                const T cur = me.tau;
                const size_t j = (size_t)x + (size_t)nx * z;
                T best = T(INFINITY);
                int bq = -1;
                if constexpr (PN) {
                    const T* wj = c.wr + j;
                    static_for<N>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        constexpr int oz = Table<R>::v.z[q], ox = Table<R>::v.x[q];
                        const T cand = pt[oz + R][x - ox].tau + wj[(size_t)q * c.n];
                        if (cand < best) { best = cand; bq = q; }
                    });
                } else {
                    const int kj = me.ck / (c.nk * N);
                    const T* Wj = c.W + kj * N;
                    static_for<N>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        constexpr int oz = Table<R>::v.z[q], ox = Table<R>::v.x[q];
                        const Cell<T> ci = pt[oz + R][x - ox];
                        const T cand = ci.tau + Wj[ci.ck + q];
                        if (cand < best) { best = cand; bq = q; }
                    });
                }
                if (best < cur) {
                    tau[j] = best;
                    changed = true;
                    c.stamp[(z / kTile) * c.TX + x / kTile] = pass;
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

// ---- row-class path --------------------------------------------------------
// When every lattice row holds one class (flat layers, the paper's layered
// models), the weight of an edge depends only on the rows of its two ends:
// w_q(z) = W[k(z - o_z)][k(z)][q].  Then
//   * in a row sweep and in the verification pass every thread of a line reads
//     the same weights (one broadcast per shared load), at offsets in the
//     class-pair table fixed per line;
//   * in a column sweep each thread owns one depth z for the whole sweep, so
//     its weight offsets are fixed per sweep;
//   * the ring holds tau only, so a pull is a 4-byte (8-byte in double)
//     shared load of tau and an independent load of the weight, an add and a
//     min -- the class loads of the class-pair path, and the weight load that
//     had to wait for them, are gone.
// Same pulls in the same order with the same rounded weights as the class-
// pair path, so the fields and parents are bit-identical.

__device__ __forceinline__ int row_class(const int* rowk, int z, int nz, int fallback) {
    return (z >= 0 && z < nz) ? rowk[z] : fallback;
}

// One node of a line per thread (lines of at most 512 nodes): the row-class
// sweep and verification written for that case, which the compiler
// schedules better than the general forms below at PPT = 1.
template <typename T, int R, int AXIS, int DIR>
__device__ void sweep_rows1(const Ctx<T>& c, T* __restrict__ tau, int pass, int since) {
    constexpr int N = Stencil<R>::N;
    const int n_lines = AXIS == 0 ? c.nz : c.nx;
    const int len = AXIS == 0 ? c.nx : c.nz;
    const int nx = c.nx, nk = c.nk;
    const int u = threadIdx.x;
    T* ring = reinterpret_cast<T*>(c.ring);
    for (int i = u; i < 8 * c.LS; i += blockDim.x) ring[i] = T(INFINITY);
    __syncthreads();
    // wo[oz + R]: offset in W of the class pair (row of i = j - o, row of j)
    // for the entries with z component oz.  Column sweeps: fixed per thread
    // (its depth z = u); row sweeps: fixed per line, the same for all threads.
    int wo[2 * R + 1];
    auto set_wo = [&](int zj) {
        const int kj = row_class(c.rowk, zj, c.nz, 0);
#pragma unroll
        for (int d = -R; d <= R; ++d) wo[d + R] = c.rowoff[zj - d] + kj * N;
    };
    if constexpr (AXIS == 1) set_wo(u < len ? u : 0);
    // Column sweeps: the thread's depth, and so each of its pulls' weights,
    // is fixed for the whole sweep; they are read once into registers (the
    // entries of the other sweep direction are never read).
    [[maybe_unused]] T wreg[N];
    if constexpr (AXIS == 1) {
        static_for<N>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr int ox = Table<R>::v.x[q], oz = Table<R>::v.z[q];
            if constexpr (ox * DIR > 0) wreg[q] = c.W[wo[oz + R] + q];
        });
    }
    auto gidx = [&](int line) {
        return AXIS == 0 ? (size_t)u + (size_t)nx * line : (size_t)line + (size_t)nx * u;
    };
    auto ring_line = [&](int line) {
        if (u < len) ring[(line & 7) * c.LS + R + u] = (line >= 0 && line < n_lines) ? tau[gidx(line)] : T(INFINITY);
    };
    bool reload = false;
    T cur = (u < len) ? tau[gidx(DIR > 0 ? 0 : n_lines - 1)] : T(INFINITY);
    for (int step = 0; step < n_lines; ++step) {
        const int line = DIR > 0 ? step : n_lines - 1 - step;
        const bool band_start = DIR > 0 ? (line % kTile == 0) : (line == n_lines - 1 || line % kTile == kTile - 1);
        if (band_start) {
            const int b = line / kTile;
            if (!band_dirty<T, AXIS>(c, b, since)) {
                const int last = DIR > 0 ? min(n_lines - 1, b * kTile + kTile - 1) : b * kTile;
                step = DIR > 0 ? last : n_lines - 1 - last;
                reload = true;
                continue;
            }
            if (reload) {
                for (int lag = 1; lag <= R; ++lag) ring_line(line - DIR * lag);
                cur = (u < len) ? tau[gidx(line)] : T(INFINITY);
                __syncthreads();
                reload = false;
            }
        }
        if constexpr (AXIS == 0) set_wo(line);
        const T nxt = (step + 1 < n_lines && u < len) ? tau[gidx(DIR > 0 ? line + 1 : line - 1)] : T(INFINITY);
        int po[R + 1];                      // ring offsets of the previous lines (32-bit shared indices)
#pragma unroll
        for (int lag = 1; lag <= R; ++lag) po[lag] = ((line - DIR * lag) & 7) * c.LS + R + u;
        const int own = (line & 7) * c.LS + R;
        if (u < len) {
            const int tx = (AXIS == 0 ? u : line) / kTile, tz = (AXIS == 0 ? line : u) / kTile;
            T best = cur;
            if (dirty(c, tx, tz, since)) {
                static_for<N>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    constexpr int oa = AXIS == 0 ? Table<R>::v.z[q] : Table<R>::v.x[q];
                    constexpr int ol = AXIS == 0 ? Table<R>::v.x[q] : Table<R>::v.z[q];
                    if constexpr (oa * DIR > 0) {
                        constexpr int lag = oa * DIR;
                        constexpr int oz = Table<R>::v.z[q];
                        if constexpr (AXIS == 1)
                            best = fmin_(best, ring[po[lag] - ol] + wreg[q]);
                        else
                            best = fmin_(best, ring[po[lag] - ol] + c.W[wo[oz + R] + q]);
                    }
                });
            }
            ring[own + u] = best;
            if (best < cur) {
                tau[gidx(line)] = best;
                c.stamp[tz * c.TX + tx] = pass;
            }
        }
        __syncthreads();
        cur = nxt;
    }
}

template <typename T, int R>
__device__ bool verify_rows1(const Ctx<T>& c, T* __restrict__ tau, int64_t src, int32_t* __restrict__ par,
                            int pass, int since) {
    constexpr int N = Stencil<R>::N;
    const int nx = c.nx, nz = c.nz, nk = c.nk;
    const int x = threadIdx.x;
    T* ring = reinterpret_cast<T*>(c.ring);
    for (int i = x; i < 16 * c.LS; i += blockDim.x) ring[i] = T(INFINITY);
    __syncthreads();
    auto store_row = [&](int row) {
        if (x < nx) ring[(row & 15) * c.LS + R + x] = (row >= 0 && row < nz) ? tau[(size_t)x + (size_t)nx * row]
                                                                              : T(INFINITY);
    };
    for (int row = 0; row < R && row < nz; ++row) store_row(row);
    bool changed = false, reload = false;
    for (int z = 0; z < nz; ++z) {
        if (z % kTile == 0) {
            const int b = z / kTile;
            if (!band_dirty<T, 0>(c, b, since)) {
                z = min(nz, z + kTile) - 1;
                reload = true;
                continue;
            }
            if (reload) {
                for (int row = z - R; row < z + R; ++row) store_row(row);
                reload = false;
            }
        }
        store_row(z + R);
        __syncthreads();
        int po[2 * R + 1], wo[2 * R + 1];   // ring offsets of rows z - d, weight-table offsets
        const int kj = c.rowk[z];
#pragma unroll
        for (int d = -R; d <= R; ++d) {
            po[d + R] = ((z - d) & 15) * c.LS + R + x;
            wo[d + R] = c.rowoff[z - d] + kj * N;
        }
        if (x < nx && dirty(c, x / kTile, z / kTile, since)) {
            const T cur = ring[po[R]];
            const size_t j = (size_t)x + (size_t)nx * z;
            T best = T(INFINITY);
            int bq = -1;
            static_for<N>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                constexpr int oz = Table<R>::v.z[q], ox = Table<R>::v.x[q];
                const T cand = ring[po[oz + R] - ox] + c.W[wo[oz + R] + q];
                if (cand < best) { best = cand; bq = q; }
            });
            if (best < cur) {
                tau[j] = best;
                changed = true;
                c.stamp[(z / kTile) * c.TX + x / kTile] = pass;
            } else if (par) {
                int32_t pj;
                if ((int64_t)j == src) pj = (int32_t)src;
                else if (isinf(cur) || bq < 0) pj = -1;
                else pj = (int32_t)((long long)j - ((long long)c.sz[bq] * nx + c.sx[bq]));
                par[j] = pj;
            }
        }
    }
    return __syncthreads_or(changed);
}

// Several adjacent nodes of a line per thread: thread t takes nodes
// PPT*t .. PPT*t + PPT-1.  The pulls of a thread's nodes from one previous
// line read overlapping windows of that line in the ring (offsets -R..R of
// each node), and in row sweeps and the verification the same weight serves
// all of them, so the unrolled loop loads each ring cell and each weight once
// for the PPT nodes: about (2R + PPT) + 2R + 1 shared loads per PPT (2R + 1)
// pulls, against two per pull with one node a thread.  Same pulls, in the same
// order per node, same rounding: fields and parents are bit-identical.
template <typename T, int R, int PPT, int AXIS, int DIR>
__device__ void sweep_rows(const Ctx<T>& c, T* __restrict__ tau, int pass, int since) {
    constexpr int N = Stencil<R>::N;
    const int n_lines = AXIS == 0 ? c.nz : c.nx;
    const int len = AXIS == 0 ? c.nx : c.nz;
    const int nx = c.nx;
    const int tid = threadIdx.x, bd = blockDim.x;
    const int u0 = PPT * tid;                       // the thread's first node
    T* ring = reinterpret_cast<T*>(c.ring);
    for (int i = tid; i < 8 * c.LS; i += bd) ring[i] = T(INFINITY);
    __syncthreads();
    // wo[p][oz + R]: offset in W of the class pair (row of i = j - o, row of j)
    // for the entries with z component oz.  Column sweeps: fixed per node for
    // the whole sweep (depth z = u0 + p); row sweeps: fixed per line, the same
    // for every node of the line (kept in wo[0]).
    constexpr int NW = AXIS == 1 ? PPT : 1;
    int wo[NW][2 * R + 1];
    auto set_wo = [&](int slot, int zj) {
        const int kj = row_class(c.rowk, zj, c.nz, 0);
#pragma unroll
        for (int d = -R; d <= R; ++d) wo[slot][d + R] = c.rowoff[zj - d] + kj * N;
    };
    if constexpr (AXIS == 1) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) set_wo(p, min(u0 + p, len - 1));
    }
    auto gidx = [&](int line, int u) {
        return AXIS == 0 ? (size_t)u + (size_t)nx * line : (size_t)line + (size_t)nx * u;
    };
    auto ring_line = [&](int line) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int u = u0 + p;
            if (u < len)
                ring[(line & 7) * c.LS + R + u] = (line >= 0 && line < n_lines) ? tau[gidx(line, u)] : T(INFINITY);
        }
    };
    auto load = [&](int line, T* t) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int u = u0 + p;
            t[p] = u < len ? tau[gidx(line, u)] : T(INFINITY);
        }
    };
    bool reload = false;
    T cur[PPT];
    load(DIR > 0 ? 0 : n_lines - 1, cur);
    for (int step = 0; step < n_lines; ++step) {
        const int line = DIR > 0 ? step : n_lines - 1 - step;
        const bool band_start = DIR > 0 ? (line % kTile == 0) : (line == n_lines - 1 || line % kTile == kTile - 1);
        if (band_start) {
            const int b = line / kTile;
            if (!band_dirty<T, AXIS>(c, b, since)) {
                const int last = DIR > 0 ? min(n_lines - 1, b * kTile + kTile - 1) : b * kTile;
                step = DIR > 0 ? last : n_lines - 1 - last;
                reload = true;
                continue;
            }
            if (reload) {
                for (int lag = 1; lag <= R; ++lag) ring_line(line - DIR * lag);
                load(line, cur);
                __syncthreads();
                reload = false;
            }
        }
        if constexpr (AXIS == 0) set_wo(0, line);
        T nxt[PPT];
        if (step + 1 < n_lines) load(DIR > 0 ? line + 1 : line - 1, nxt);
        const int own = (line & 7) * c.LS + R;
        if (u0 < len) {
            int po[R + 1];                  // ring offsets of the thread's first node in the previous lines
#pragma unroll
            for (int lag = 1; lag <= R; ++lag) po[lag] = ((line - DIR * lag) & 7) * c.LS + R + u0;
            // the thread's nodes share their tile (PPT divides the tile width)
            const int tx = (AXIS == 0 ? u0 : line) / kTile, tz = (AXIS == 0 ? line : u0) / kTile;
            T best[PPT];
#pragma unroll
            for (int p = 0; p < PPT; ++p) best[p] = cur[p];
            if (dirty(c, tx, tz, since)) {
                static_for<N>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    constexpr int oa = AXIS == 0 ? Table<R>::v.z[q] : Table<R>::v.x[q];
                    constexpr int ol = AXIS == 0 ? Table<R>::v.x[q] : Table<R>::v.z[q];
                    if constexpr (oa * DIR > 0) {
                        constexpr int lag = oa * DIR;
                        constexpr int oz = Table<R>::v.z[q];
                        if constexpr (AXIS == 0) {
                            const T w = c.W[wo[0][oz + R] + q];
#pragma unroll
                            for (int p = 0; p < PPT; ++p) best[p] = fmin_(best[p], ring[po[lag] + p - ol] + w);
                        } else {
#pragma unroll
                            for (int p = 0; p < PPT; ++p)
                                best[p] = fmin_(best[p], ring[po[lag] + p - ol] + c.W[wo[p][oz + R] + q]);
                        }
                    }
                });
            }
            bool touched = false;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const int u = u0 + p;
                if (u < len) {
                    ring[own + u] = best[p];
                    if (best[p] < cur[p]) {
                        tau[gidx(line, u)] = best[p];
                        touched = true;
                    }
                }
            }
            if (touched) c.stamp[tz * c.TX + tx] = pass;
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < PPT; ++p) cur[p] = nxt[p];
    }
}

// Verification pass of the row-class path: rows, a 16-row ring of tau; the
// weights of the row's in-neighbours are read from the class-pair table at
// addresses that are the same for every thread (one broadcast per load) and
// serve the thread's PPT adjacent nodes.
template <typename T, int R, int PPT>
__device__ bool verify_rows(const Ctx<T>& c, T* __restrict__ tau, int64_t src, int32_t* __restrict__ par,
                            int pass, int since) {
    constexpr int N = Stencil<R>::N;
    const int nx = c.nx, nz = c.nz;
    const int tid = threadIdx.x, bd = blockDim.x;
    const int x0 = PPT * tid;
    T* ring = reinterpret_cast<T*>(c.ring);
    for (int i = tid; i < 16 * c.LS; i += bd) ring[i] = T(INFINITY);
    __syncthreads();
    auto store_row = [&](int row) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int x = x0 + p;
            if (x < nx)
                ring[(row & 15) * c.LS + R + x] = (row >= 0 && row < nz) ? tau[(size_t)x + (size_t)nx * row] : T(INFINITY);
        }
    };
    for (int row = 0; row < R && row < nz; ++row) store_row(row);
    bool changed = false, reload = false;
    for (int z = 0; z < nz; ++z) {
        if (z % kTile == 0) {
            const int b = z / kTile;
            if (!band_dirty<T, 0>(c, b, since)) {
                z = min(nz, z + kTile) - 1;
                reload = true;
                continue;
            }
            if (reload) {
                for (int row = z - R; row < z + R; ++row) store_row(row);
                reload = false;
            }
        }
        store_row(z + R);
        __syncthreads();
        if (x0 < nx && dirty(c, x0 / kTile, z / kTile, since)) {
            int wo[2 * R + 1], po[2 * R + 1];   // weight-table offsets and ring offsets of the rows z - d
            const int kj = c.rowk[z];
#pragma unroll
            for (int d = -R; d <= R; ++d) {
                wo[d + R] = c.rowoff[z - d] + kj * N;
                po[d + R] = ((z - d) & 15) * c.LS + R + x0;
            }
            T best[PPT];
            int bq[PPT];
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                best[p] = T(INFINITY);
                bq[p] = -1;
            }
            static_for<N>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                constexpr int oz = Table<R>::v.z[q], ox = Table<R>::v.x[q];
                const T w = c.W[wo[oz + R] + q];
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    const T cand = ring[po[oz + R] + p - ox] + w;
                    if (cand < best[p]) { best[p] = cand; bq[p] = q; }
                }
            });
            bool touched = false;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const int x = x0 + p;
                if (x >= nx) continue;
                const T cur = ring[po[R] + p];
                const size_t j = (size_t)x + (size_t)nx * z;
                if (best[p] < cur) {
                    tau[j] = best[p];
                    touched = true;
                } else if (par) {
                    int32_t pj;
                    if ((int64_t)j == src) pj = (int32_t)src;
                    else if (isinf(cur) || bq[p] < 0) pj = -1;
                    else pj = (int32_t)((long long)j - ((long long)c.sz[bq[p]] * nx + c.sx[bq[p]]));
                    par[j] = pj;
                }
            }
            if (touched) {
                changed = true;
                c.stamp[(z / kTile) * c.TX + x0 / kTile] = pass;
            }
        }
    }
    return __syncthreads_or(changed);
}

// One field component (field, comp) of one lattice, by the CTA.
template <typename T, int R, int PPT, bool PN>
__device__ __forceinline__ void relax_fast_field(const Args& a, int field, int comp) {
    constexpr int N = Stencil<R>::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = a.n_classes;
    const int mode = field % a.n_modes;
    const int s = field / a.n_modes;
    const int line_max = max(a.nx, a.nz);
    Ctx<T> c;
    c.nx = a.nx; c.nz = a.nz; c.nk = nk;
    c.n = (size_t)a.nx * a.nz;
    c.TX = (a.nx + kTile - 1) / kTile;
    c.TZ = (a.nz + kTile - 1) / kTile;
    c.LS = ((line_max + 2 * R) + 3) & ~3;
    unsigned char* p = smem_raw;
    c.W = reinterpret_cast<T*>(p); p += PN ? 0 : (size_t)nk * nk * N * sizeof(T);
    c.ring = reinterpret_cast<Cell<T>*>(p); p += (size_t)16 * c.LS * sizeof(Cell<T>);
    c.stamp = reinterpret_cast<int*>(p); p += (size_t)c.TX * c.TZ * sizeof(int);
    c.sx = reinterpret_cast<short*>(p); p += N * sizeof(short);
    c.sz = reinterpret_cast<short*>(p); p += N * sizeof(short);
    int* rowk_s = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(p) + 3) & ~uintptr_t(3));
    c.rowk = rowk_s;
    int* rowoff_s = rowk_s + a.nz;              // [nz + 2R], entry z + R for row z
    c.rowoff = rowoff_s + R;
    c.wr = PN ? static_cast<const T*>(a.wrow) + (size_t)(mode * 2 + comp) * N * c.n : nullptr;
    c.wc = PN ? static_cast<const T*>(a.wcol) + (size_t)(mode * 2 + comp) * N * c.n : nullptr;

    if (threadIdx.x == 0)
        static_for<N>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr short vx = Table<R>::v.x[q], vz = Table<R>::v.z[q];
            c.sx[q] = vx;
            c.sz[q] = vz;
        });
    for (int t = threadIdx.x; t < c.TX * c.TZ; t += blockDim.x) c.stamp[t] = 0;
    __syncthreads();
    if constexpr (!PN) {
        const T* sel = static_cast<const T*>(comp == 0 ? a.Vsel : a.Asel) + (size_t)mode * nk * a.n_off;
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
    }

    T* tau = static_cast<T*>(comp == 0 ? a.tauR : a.tauI) + (size_t)field * c.n;
    int32_t* par = comp == 0 ? a.parR : a.parI;
    if (par) par += (size_t)field * c.n;
    const int64_t src = a.src[s];
    for (size_t j = threadIdx.x; j < c.n; j += blockDim.x) tau[j] = (j == (size_t)src) ? T(0) : T(INFINITY);
    __syncthreads();

    // Row-class path: every row one class (checked on the row classes that
    // row_classes_kernel wrote).
    bool rows = false;
    if constexpr (!PN) {
        if (a.rowk) {
            bool ok = true;
            for (int z = threadIdx.x; z < a.nz; z += blockDim.x) {
                const int k = a.rowk[z];
                rowk_s[z] = k;
                ok = ok && k >= 0 && k < nk;
            }
            rows = __syncthreads_and(ok);
            if (rows) {
                for (int z = (int)threadIdx.x - R; z < a.nz + R; z += blockDim.x)
                    rowoff_s[z + R] = (z >= 0 && z < a.nz) ? rowk_s[z] * nk * N : 0;
                __syncthreads();
            }
        }
    }

    // pass numbers start at 1; every tile starts dirty (stamp 0 >= last 0)
    int pass = 1;
    int last[5] = {0, 0, 0, 0, 0};
    int used = -1;
    if constexpr (!PN) {
        if (rows) {
            for (int cycle = 0; cycle < a.max_cycles; ++cycle) {
                bool changed;
                if constexpr (PPT == 1) {
                    sweep_rows1<T, R, 0, +1>(c, tau, pass, last[0]); last[0] = pass++;
                    sweep_rows1<T, R, 1, +1>(c, tau, pass, last[1]); last[1] = pass++;
                    sweep_rows1<T, R, 1, -1>(c, tau, pass, last[2]); last[2] = pass++;
                    sweep_rows1<T, R, 0, -1>(c, tau, pass, last[3]); last[3] = pass++;
                    changed = verify_rows1<T, R>(c, tau, src, par, pass, last[4]);
                } else {
                    sweep_rows<T, R, PPT, 0, +1>(c, tau, pass, last[0]); last[0] = pass++;
                    sweep_rows<T, R, PPT, 1, +1>(c, tau, pass, last[1]); last[1] = pass++;
                    sweep_rows<T, R, PPT, 1, -1>(c, tau, pass, last[2]); last[2] = pass++;
                    sweep_rows<T, R, PPT, 0, -1>(c, tau, pass, last[3]); last[3] = pass++;
                    changed = verify_rows<T, R, PPT>(c, tau, src, par, pass, last[4]);
                }
                last[4] = pass++;
                if (!changed) {
                    used = cycle + 1;
                    break;
                }
            }
            if (threadIdx.x == 0) a.status[field * 2 + comp] = used;
            return;
        }
    }
    for (int cycle = 0; cycle < a.max_cycles; ++cycle) {
        sweep<T, R, PPT, 0, +1, PN>(c, tau, a.cls, pass, last[0]); last[0] = pass++;
        sweep<T, R, PPT, 1, +1, PN>(c, tau, a.cls, pass, last[1]); last[1] = pass++;
        sweep<T, R, PPT, 1, -1, PN>(c, tau, a.cls, pass, last[2]); last[2] = pass++;
        sweep<T, R, PPT, 0, -1, PN>(c, tau, a.cls, pass, last[3]); last[3] = pass++;
        const bool changed = verify<T, R, PPT, PN>(c, tau, a.cls, src, par, pass, last[4]);
        last[4] = pass++;
        if (!changed) {
            used = cycle + 1;
            break;
        }
    }
    if (threadIdx.x == 0) a.status[field * 2 + comp] = used;
}

template <typename T, int R, int PPT, bool PN>
__global__ void __launch_bounds__(512, PPT == 1 && sizeof(T) == 4 ? 2 : 1) relax_fast_kernel(Args a) {
    // Attenuation fields (several sweep cycles) launch first and propagation
    // fields (mostly one cycle) fill the tail of the grid.
    const int n_fields = gridDim.x >> 1;
    const int comp = (int)blockIdx.x < n_fields ? 1 : 0;
    const int field = comp ? (int)blockIdx.x : (int)blockIdx.x - n_fields;
    relax_fast_field<T, R, PPT, PN>(a, field, comp);
}

// Several 2D lattices of one launch shape (stencil, nodes a thread, weight
// form) in one persistent launch.  The work items are the field components
// of every lattice: first the attenuation components of all lattices, then
// the propagation ones (each lattice's in turn, largest lattice first; the
// host orders the table).  Each CTA claims the next item from a device counter
// (zeroed before the launch) until none is left, and relaxes it with its
// lattice's arguments, read in place from the table (a kernel parameter).
// The block is sized for the longest line of the batch and the shared memory
// for its largest lattice.  With one node a thread the kernel is held to 64
// registers, two CTAs an SM, as the single-lattice kernel chooses by itself
// (a few bytes of spills); with 2 or 4 it keeps 128, no spills.
constexpr int kMaxFastLattices = 24;

struct FastTable {
    int n;
    long long start[2 * kMaxFastLattices + 1];   // item ranges: attenuation of lattice l at start[l], propagation at start[n + l]
    Args a[kMaxFastLattices];
};

template <typename T, int R, int PPT, bool PN>
__global__ void __launch_bounds__(512, PPT == 1 ? 2 : 1) relax_fast_multi_kernel(const __grid_constant__ FastTable t,
                                                               unsigned long long* counter) {
    __shared__ long long s_item;
    const long long total = t.start[2 * t.n];
    for (;;) {
        __syncthreads();                      // the previous item's shared memory is no longer read
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        int r = 0;
        while (r + 1 < 2 * t.n && t.start[r + 1] <= item) ++r;
        const int l = r < t.n ? r : r - t.n;
        relax_fast_field<T, R, PPT, PN>(t.a[l], (int)(item - t.start[r]), r < t.n ? 1 : 0);
    }
}

}  // namespace fast
}  // namespace chert
