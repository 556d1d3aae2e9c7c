// Direction lookup (Eq. 27-28), traveltime relaxation (Eq. 29-31), parents and
// raypaths (Eq. 33-34) on a 2D node lattice.
//
// Relaxation.  The fixed point tau_j = min(tau_j, min_i tau_i + w_ij) of Eq. 31
// is unique (all weights are >= 0), so any order of relaxations that runs to
// convergence returns it exactly.  One CTA owns one (source, mode, component)
// field and relaxes it in sweep order: a cycle pulls every node from its
// in-neighbours on earlier lines of four sweeps -- rows top-down (offsets with
// o_z > 0), columns left-to-right (o_x > 0), columns right-to-left (o_x < 0),
// rows bottom-up (o_z < 0).  Every offset falls in at least one sweep, no node
// is written by two threads, and a line only reads lines finished before it,
// so no atomics are needed; the last R+1 lines of tau and class ids live in a
// shared-memory ring.  A verification pass then pulls each node from all of its
// in-neighbours: if nothing improves the field is the fixed point and the same
// pass has produced the parents par_j = argmin_i (tau_i + w_ij) (ties to the
// smallest i); otherwise another cycle runs.  Weights come from a per-CTA
// table W[o][k_i][k_j] in shared memory built from the lookup.
#include <math.h>
#include <stdint.h>

#include <limits.h>

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "ff.cuh"
#include "relax_fast.cuh"
#include "relax_frontier.cuh"

namespace chert {
namespace {

constexpr int kMaxOff = 512;

struct Offsets {
    int n;
    short x[kMaxOff], y[kMaxOff], z[kMaxOff];
};

// ------------------------------------------------------------ lookup kernel
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }

// One warp per (mode, class, offset): argmax of d.r over the class's entries.
template <typename T>
__global__ void edge_table_kernel(const T* __restrict__ rx, const T* __restrict__ ry, const T* __restrict__ rz,
                                  const T* __restrict__ V, const T* __restrict__ A,
                                  const uint8_t* __restrict__ flag, int n_modes, int n_classes,
                                  int n_dir, Offsets off, int32_t* __restrict__ idx_out,
                                  T* __restrict__ Vsel, T* __restrict__ Asel) {
    const int lane = threadIdx.x & 31;
    const long long w = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const long long total = static_cast<long long>(n_modes) * n_classes * off.n;
    if (w >= total) return;
    const int o = static_cast<int>(w % off.n);
    const long long mk = w / off.n;                  // mode * n_classes + class
    const double ox = off.x[o], oy = off.y[o], oz = off.z[o];
    const T nrm = T(sqrt(ox * ox + oy * oy + oz * oz));
    const T dx = div_rn(T(ox), nrm), dy = div_rn(T(oy), nrm), dz = div_rn(T(oz), nrm);
    const size_t base = static_cast<size_t>(mk) * n_dir;
    T best = T(-INFINITY);
    int bi = -1;
    for (int e = lane; e < n_dir; e += 32) {
        if (flag[base + e]) continue;
        T dot = mul_rn(dx, rx[base + e]);
        if (ry) dot = add_rn(dot, mul_rn(dy, ry[base + e]));
        dot = add_rn(dot, mul_rn(dz, rz[base + e]));
        if (dot > best) { best = dot; bi = e; }     // increasing e: first max kept
    }
    for (int s = 16; s > 0; s >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, s);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, s);
        if (oi >= 0 && (bi < 0 || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
    }
    if (lane == 0) {
        const size_t out = static_cast<size_t>(mk) * off.n + o;
        idx_out[out] = bi;
        Vsel[out] = bi >= 0 ? V[base + bi] : T(NAN);
        Asel[out] = bi >= 0 ? A[base + bi] : T(NAN);
    }
}

// ------------------------------------------------------------ relaxation
struct FieldArgs {
    int nx, nz, n_classes, n_modes, n_sources, max_cycles, ring;
    int ny;                      // 1 for 2D lattices
    double dx;
    const int32_t* cls;
    const int64_t* src;
    void *tauR, *tauI;
    int32_t *parR, *parI;
    const void *Vsel, *Asel;     // [n_modes][n_classes][n_off]
    int* status;                 // [field*2 + component]: cycles used, -1 = cap hit
    // 3D: CTAs per field component (parts) and their barrier words, kSyncStride
    // unsigned per field component (barrier count, two change flags), zeroed
    // before the launch; parts > 1 only under a cooperative launch
    int parts;
    unsigned* sync;
    // 3D: the offsets are the standard reach-2 table (Stencil3) in its order
    int std3;
};

template <typename T>
__device__ __forceinline__ T edge_w(int comp, T L, T a, T b) {
    // Eq. 29-30 with the segment averages of Eq. 28
    return comp == 0 ? div_rn(L, mul_rn(T(0.5), add_rn(a, b))) : mul_rn(L, mul_rn(T(0.5), add_rn(a, b)));
}

// Class ids index shared-memory tables, so every load is clamped into range;
// check_classes_kernel reports out-of-range ids as an argument error.
__device__ __forceinline__ int clamp_class(int k, int nk) { return min(max(k, 0), nk - 1); }

__global__ void check_classes_kernel(const int32_t* __restrict__ cls, long long n, int nk, int* bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (cls[i] < 0 || cls[i] >= nk) { atomicOr(bad, 1); return; }
}

// Shared memory layout of relax_kernel.
template <typename T>
struct Smem {
    T* W;          // [n_off][nk][nk] (table) or [nk][n_off] raw values
    T* L;          // [n_off]
    T* ring;       // [ring][line_max]
    int32_t* cring;  // [ring][line_max]
    short* lists;  // 4 x [n_off] offset indices per sweep
    int* counts;   // 4
};

// Weight of the edge i -> j through offset o (Eq. 28-30):
//   WMODE 1: pair table W[o][k_i][k_j] in shared memory;
//   WMODE 0: looked-up values [k][o] in shared memory, formula per pull;
//   WMODE 2: looked-up values [k][o] in global memory (any number of classes,
//            e.g. one class per cell), formula per pull.
template <typename T, int WMODE>
__device__ __forceinline__ T pull_weight(const Smem<T>& sm, const T* __restrict__ gsel, int n_off, int nk,
                                         int comp, int o, int ki, int kj) {
    if (WMODE == 1) return sm.W[(o * nk + ki) * nk + kj];
    if (WMODE == 0) return edge_w<T>(comp, sm.L[o], sm.W[ki * n_off + o], sm.W[kj * n_off + o]);
    return edge_w<T>(comp, sm.L[o], gsel[(size_t)ki * n_off + o], gsel[(size_t)kj * n_off + o]);
}

// One sweep: lines advance along `axis` (0: rows in z, 1: columns in x) in
// direction `dir`; each node pulls from the offsets of its sweep list.
template <typename T, int WMODE>
__device__ bool sweep(const Smem<T>& sm, const T* __restrict__ gsel, const Offsets& off, int list, int axis,
                      int dir, T* tau, const int32_t* __restrict__ cls, int nx, int nz, int nk, int comp,
                      int ring) {
    const int n_lines = axis == 0 ? nz : nx;
    const int len = axis == 0 ? nx : nz;
    const short* lst = sm.lists + list * off.n;
    const int cnt = sm.counts[list];
    bool changed = false;
    for (int step = 0; step < n_lines; ++step) {
        const int line = dir > 0 ? step : n_lines - 1 - step;
        const int slot = line % ring;
        for (int u = threadIdx.x; u < len; u += blockDim.x) {
            const size_t j = axis == 0 ? (size_t)u + (size_t)nx * line : (size_t)line + (size_t)nx * u;
            const T cur = tau[j];
            const int kj = clamp_class(cls[j], nk);
            sm.cring[slot * len + u] = kj;
            T best = cur;
            for (int q = 0; q < cnt; ++q) {
                const int o = lst[q];
                const int oa = axis == 0 ? off.z[o] : off.x[o];   // across-line component
                const int ol = axis == 0 ? off.x[o] : off.z[o];   // along-line component
                const int il = line - oa;
                const int iu = u - ol;
                if (il < 0 || il >= n_lines || iu < 0 || iu >= len) continue;
                const int s = (il % ring) * len + iu;
                const int ki = sm.cring[s];
                const T w = pull_weight<T, WMODE>(sm, gsel, off.n, nk, comp, o, ki, kj);
                best = fmin(best, sm.ring[s] + w);
            }
            sm.ring[slot * len + u] = best;
            if (best < cur) {
                tau[j] = best;
                changed = true;
            }
        }
        __syncthreads();
    }
    return __syncthreads_or(changed);
}

// Pull every node from all in-neighbours; lower tau where possible (returns
// true if anything changed) and record the argmin parent.
template <typename T, int WMODE>
__device__ bool verify(const Smem<T>& sm, const T* __restrict__ gsel, const Offsets& off, T* tau,
                       const int32_t* __restrict__ cls, int nx, int nz, int nk, int comp, int64_t src,
                       int32_t* par) {
    bool changed = false;
    const int n = nx * nz;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int xj = j % nx, zj = j / nx;
        const int kj = clamp_class(cls[j], nk);
        const T cur = tau[j];
        T best = T(INFINITY);
        int bi = -1;
        for (int o = 0; o < off.n; ++o) {
            const int xi = xj - off.x[o], zi = zj - off.z[o];
            if (xi < 0 || xi >= nx || zi < 0 || zi >= nz) continue;
            const int i = xi + nx * zi;
            const T ti = tau[i];
            const int ki = clamp_class(cls[i], nk);
            const T w = pull_weight<T, WMODE>(sm, gsel, off.n, nk, comp, o, ki, kj);
            const T c = ti + w;
            if (c < best || (c == best && i < bi)) { best = c; bi = i; }
        }
        if (best < cur) {
            tau[j] = best;
            changed = true;
        } else if (par) {
            par[j] = (j == src) ? static_cast<int32_t>(src) : (isinf(cur) ? -1 : bi);
        }
    }
    return __syncthreads_or(changed);
}

template <typename T, int WMODE>
__global__ void __launch_bounds__(512) relax_kernel(FieldArgs a, Offsets off) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = a.n_classes;
    const int field = blockIdx.x >> 1;          // source * n_modes + mode
    const int comp = blockIdx.x & 1;            // 0: propagation, 1: attenuation
    const int mode = field % a.n_modes;
    const int s = field / a.n_modes;
    const int line_max = max(a.nx, a.nz);
    const size_t n = static_cast<size_t>(a.nx) * a.nz;

    Smem<T> sm;
    unsigned char* p = smem_raw;
    const size_t wcount = WMODE == 1 ? static_cast<size_t>(off.n) * nk * nk
                          : WMODE == 0 ? static_cast<size_t>(nk) * off.n : 0;
    sm.W = reinterpret_cast<T*>(p); p += wcount * sizeof(T);
    sm.L = reinterpret_cast<T*>(p); p += off.n * sizeof(T);
    sm.ring = reinterpret_cast<T*>(p); p += static_cast<size_t>(a.ring) * line_max * sizeof(T);
    sm.cring = reinterpret_cast<int32_t*>(p); p += static_cast<size_t>(a.ring) * line_max * 4;
    sm.lists = reinterpret_cast<short*>(p); p += 4 * off.n * sizeof(short);
    sm.counts = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(p) + 3) & ~uintptr_t(3));

    // weights of this (mode, component)
    const T* sel = static_cast<const T*>(comp == 0 ? a.Vsel : a.Asel) +
                   static_cast<size_t>(mode) * nk * off.n;
    for (int o = threadIdx.x; o < off.n; o += blockDim.x) {
        const double ox = off.x[o], oz = off.z[o];
        sm.L[o] = T(a.dx * sqrt(ox * ox + oz * oz));
    }
    __syncthreads();
    if (WMODE == 1) {
        for (int t = threadIdx.x; t < off.n * nk * nk; t += blockDim.x) {
            const int kj = t % nk, ki = (t / nk) % nk, o = t / (nk * nk);
            sm.W[t] = edge_w<T>(comp, sm.L[o], sel[ki * off.n + o], sel[kj * off.n + o]);
        }
    } else if (WMODE == 0) {
        for (int t = threadIdx.x; t < nk * off.n; t += blockDim.x) sm.W[t] = sel[t];
    }
    if (threadIdx.x == 0) {
        int c[4] = {0, 0, 0, 0};
        for (int o = 0; o < off.n; ++o) {
            if (off.z[o] > 0) sm.lists[0 * off.n + c[0]++] = (short)o;   // rows, top-down
            if (off.x[o] > 0) sm.lists[1 * off.n + c[1]++] = (short)o;   // columns, left-right
            if (off.x[o] < 0) sm.lists[2 * off.n + c[2]++] = (short)o;   // columns, right-left
            if (off.z[o] < 0) sm.lists[3 * off.n + c[3]++] = (short)o;   // rows, bottom-up
        }
        for (int i = 0; i < 4; ++i) sm.counts[i] = c[i];
    }

    T* tau = static_cast<T*>(comp == 0 ? a.tauR : a.tauI) + static_cast<size_t>(field) * n;
    int32_t* par = comp == 0 ? a.parR : a.parI;
    if (par) par += static_cast<size_t>(field) * n;
    const int64_t src = a.src[s];
    for (size_t j = threadIdx.x; j < n; j += blockDim.x) tau[j] = (j == (size_t)src) ? T(0) : T(INFINITY);
    __syncthreads();

    int used = -1;
    for (int cycle = 0; cycle < a.max_cycles; ++cycle) {
        sweep<T, WMODE>(sm, sel, off, 0, 0, +1, tau, a.cls, a.nx, a.nz, nk, comp, a.ring);
        sweep<T, WMODE>(sm, sel, off, 1, 1, +1, tau, a.cls, a.nx, a.nz, nk, comp, a.ring);
        sweep<T, WMODE>(sm, sel, off, 2, 1, -1, tau, a.cls, a.nx, a.nz, nk, comp, a.ring);
        sweep<T, WMODE>(sm, sel, off, 3, 0, -1, tau, a.cls, a.nx, a.nz, nk, comp, a.ring);
        if (!verify<T, WMODE>(sm, sel, off, tau, a.cls, a.nx, a.nz, nk, comp, src, par)) {
            used = cycle + 1;
            break;
        }
    }
    if (threadIdx.x == 0) a.status[blockIdx.x] = used;
}

// ------------------------------------------------------------ frontier label correcting
// (scheduler 3; see relax_frontier.cuh).  Shared memory: the class-pair weight
// table [n_off][nk][nk], then the two frontier bitmaps.
template <typename T>
__global__ void __launch_bounds__(1024) relax_frontier_kernel(frontier::Args a, Offsets off) {
    using B = frontier::Bits<T>;
    using U = typename B::U;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = a.n_classes;
    const int nx = a.nx, nz = a.nz;
    const int n = nx * nz;
    const int fc = blockIdx.x, field = fc >> 1, comp = fc & 1;
    const int mode = field % a.n_modes, s = field / a.n_modes;
    const int nwords = (n + 31) >> 5;
    T* W = reinterpret_cast<T*>(smem_raw);
    unsigned* bm0 = reinterpret_cast<unsigned*>(smem_raw + (((size_t)off.n * nk * nk * sizeof(T) + 15) & ~size_t(15)));
    unsigned* bm1 = bm0 + nwords;
    const T* sel = static_cast<const T*>(comp == 0 ? a.Vsel : a.Asel) + (size_t)mode * nk * off.n;
    for (int t = threadIdx.x; t < off.n * nk * nk; t += blockDim.x) {
        const int kj = t % nk, ki = (t / nk) % nk, o = t / (nk * nk);
        const double ox = off.x[o], oz = off.z[o];
        const T L = T(a.dx * sqrt(ox * ox + oz * oz));
        W[t] = edge_w<T>(comp, L, sel[ki * off.n + o], sel[kj * off.n + o]);
    }
    U* tau = reinterpret_cast<U*>(static_cast<T*>(comp == 0 ? a.tauR : a.tauI) + (size_t)field * n);
    int32_t* par = comp == 0 ? a.parR : a.parI;
    if (par) par += (size_t)field * n;
    const int64_t src = a.src[s];
    for (int j = threadIdx.x; j < n; j += blockDim.x) tau[j] = B::enc(j == src ? T(0) : T(INFINITY));
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) bm0[w] = (w == (int)(src >> 5)) ? (1u << (src & 31)) : 0u;
    __syncthreads();
    unsigned *cur = bm0, *nxt = bm1;
    int used = -1;
    for (int round = 0; round < a.max_rounds; ++round) {
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) nxt[w] = 0u;
        __syncthreads();
        // every node of the frontier pushes to all its out-neighbours: a warp
        // takes one bitmap word at a time, and for each node in it the lanes
        // share the stencil's offsets
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        for (int w = warp; w < nwords; w += nwarps) {
            unsigned bits = cur[w];
            while (bits) {
                const int i = (w << 5) + __ffs(bits) - 1;
                bits &= bits - 1;
                const T ti = B::dec(__ldcg(tau + i));
                const int xi = i % nx, zi = i / nx;
                const int ki = clamp_class(__ldg(a.cls + i), nk);
                for (int o = lane; o < off.n; o += 32) {
                    const int xj = xi + off.x[o], zj = zi + off.z[o];
                    if (xj < 0 || xj >= nx || zj < 0 || zj >= nz) continue;
                    const int j = xj + nx * zj;
                    const int kj = clamp_class(__ldg(a.cls + j), nk);
                    const U cand = B::enc(ti + W[(o * nk + ki) * nk + kj]);
                    if (cand < atomicMin(tau + j, cand)) atomicOr(nxt + (j >> 5), 1u << (j & 31));
                }
            }
        }
        bool any = false;
        __syncthreads();
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) any = any || nxt[w] != 0u;
        if (!__syncthreads_or(any)) {
            used = round + 1;
            break;
        }
        unsigned* t = cur;
        cur = nxt;
        nxt = t;
    }
    // parents, and a check that no in-neighbour improves any node
    bool bad = false;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int xj = j % nx, zj = j / nx;
        const int kj = clamp_class(__ldg(a.cls + j), nk);
        const T tj = B::dec(__ldcg(tau + j));
        T best = T(INFINITY);
        int bi = -1;
        for (int o = 0; o < off.n; ++o) {
            const int xi = xj - off.x[o], zi = zj - off.z[o];
            if (xi < 0 || xi >= nx || zi < 0 || zi >= nz) continue;
            const int i = xi + nx * zi;
            const int ki = clamp_class(__ldg(a.cls + i), nk);
            const T c = B::dec(__ldcg(tau + i)) + W[(o * nk + ki) * nk + kj];
            if (c < best || (c == best && i < bi)) { best = c; bi = i; }
        }
        if (best < tj) bad = true;
        if (par) par[j] = (j == src) ? (int32_t)src : (isinf(tj) ? -1 : bi);
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) a.status[fc] = bad ? -1 : used;
}

// ------------------------------------------------------------ block-heap marching
// The paper's block scheduler (Eq. 32): a block's key is the least traveltime
// that may still propagate from it; the block with the smallest key is taken
// next, relaxed inside (every node pulls all its in-neighbours, repeatedly,
// until nothing in the block changes), and the 3 x 3 blocks around it are
// re-keyed with the least value it lowered.  When no block is dirty, every
// block has been relaxed after its neighbours' last change: the field is the
// fixed point of Eq. 31 (the same one the sweeps reach).  The verification
// pass then writes the parents.  Blocks are 32 x 32 tiles; one CTA per field
// component; the priority queue is a block-wide argmin over the tile keys in
// shared memory (ties to the lower tile index).
constexpr int kBT = 32;

template <typename T, typename B>
__device__ __forceinline__ B to_bits(T v) {
    if constexpr (sizeof(T) == 8) return static_cast<B>(__double_as_longlong(v));
    else return static_cast<B>(__float_as_uint(v));
}
template <typename T, typename B>
__device__ __forceinline__ T from_bits(B b) {
    if constexpr (sizeof(T) == 8) return __longlong_as_double(static_cast<long long>(b));
    else return __uint_as_float(static_cast<unsigned int>(b));
}

template <typename T>
__device__ __forceinline__ void block_argmin(T v, int i, T* rv, int* ri, T& out_v, int& out_i) {
    for (int o = 16; o > 0; o >>= 1) {
        const T v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (v2 < v || (v2 == v && i2 >= 0 && (i < 0 || i2 < i))) { v = v2; i = i2; }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { rv[w] = v; ri[w] = i; }
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? rv[lane] : T(INFINITY);
        i = lane < (int)(blockDim.x >> 5) ? ri[lane] : -1;
        for (int o = 16; o > 0; o >>= 1) {
            const T v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
            if (v2 < v || (v2 == v && i2 >= 0 && (i < 0 || i2 < i))) { v = v2; i = i2; }
        }
        if (lane == 0) { rv[0] = v; ri[0] = i; }
    }
    __syncthreads();
    out_v = rv[0];
    out_i = ri[0];
    __syncthreads();
}

// Window of one block in shared memory: the block's kBT x kBT nodes and a
// halo of H nodes (the stencil's reach) on every side, H <= kBH; positions
// off the lattice hold +inf, so no pull needs a bounds check.
constexpr int kBH = 8;
// Inside a block, 8 x 8 sub-blocks record whether a node of theirs changed in
// an iteration; the next iteration re-evaluates only the nodes whose 3 x 3
// sub-block neighbourhood (which covers a reach of kBH) saw a change.  Three
// flag sets rotate: read (previous iteration), written (this one), cleared
// (the next one), so no barrier is needed between clearing and writing.
constexpr int kSB = 8, kNSB = kBT / kSB;

// One field component by block-heap marching, shared by both kernels below.
// The window of the block being relaxed is wt (SW x SW, halo H); stage(q, g,
// in) stages what the pulls need besides tau at window position q (lattice
// node g, in = on the lattice); pull(e, x, z, cur) returns the least of cur
// and the pulls of the node at window position e (lattice x, z); verify()
// is the verification pass (true: something improved).  Returns the cycles
// used (swept + verification passes), or -1 when a cap ran out.
template <typename T, typename Stage, typename Pull, typename Verify>
__device__ __forceinline__ int bhm_field(T* tau, int nx, int nz, int64_t src, int max_cycles, int swept, int H,
                                         T* key, T* rv, int* ri, T* wt, int* chg, unsigned char* m9raw,
                                         Stage stage, Pull pull, Verify verify_pass) {
    using Bits = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
    Bits* m9 = reinterpret_cast<Bits*>(m9raw);
    const size_t n = static_cast<size_t>(nx) * nz;
    const int TX = (nx + kBT - 1) / kBT, TZ = (nz + kBT - 1) / kBT, nt = TX * TZ;
    const int SW = kBT + 2 * H;
    for (size_t j = threadIdx.x; j < n; j += blockDim.x) tau[j] = (j == (size_t)src) ? T(0) : T(INFINITY);
    for (int t = threadIdx.x; t < nt; t += blockDim.x)
        key[t] = t == (int)((src % nx) / kBT + (src / nx) / kBT * TX) ? T(0) : T(INFINITY);
    __syncthreads();

    const long long max_pops = (long long)max_cycles * nt * 8;
    long long pops = 0;
    for (int cycle = 0; cycle < max_cycles && pops <= max_pops; ++cycle) {
        for (;;) {
            T bv = T(INFINITY);
            int bi = -1;
            for (int t = threadIdx.x; t < nt; t += blockDim.x)
                if (key[t] < bv) { bv = key[t]; bi = t; }
            T kv;
            int kt;
            block_argmin(bv, bi, rv, ri, kv, kt);
            if (kt < 0 || ++pops > max_pops) break;
            const int x0 = (kt % TX) * kBT, z0 = (kt / TX) * kBT;
            for (int q = threadIdx.x; q < SW * SW; q += blockDim.x) {      // stage the window
                const int x = x0 - H + q % SW, z = z0 - H + q / SW;
                const bool in = x >= 0 && x < nx && z >= 0 && z < nz;
                const size_t g = in ? (size_t)x + (size_t)nx * z : 0;
                wt[q] = in ? tau[g] : T(INFINITY);
                stage(q, g, in);
            }
            if (threadIdx.x == 0) key[kt] = T(INFINITY);
            for (int t = threadIdx.x; t < 3 * kNSB * kNSB; t += blockDim.x) chg[t] = 0;
            if (threadIdx.x < 9) m9[threadIdx.x] = to_bits<T, Bits>(T(INFINITY));
            __syncthreads();
            unsigned changed = 0;                            // bit k: node threadIdx.x + k * blockDim.x
            bool still = false;
            for (int it = 0; it < 4 * kBT; ++it) {          // relax the block to local convergence
                bool any = false;
                const int* prev = chg + ((it + 2) % 3) * kNSB * kNSB;
                int* now = chg + (it % 3) * kNSB * kNSB;
                if (it > 0 && threadIdx.x < kNSB * kNSB) chg[((it + 1) % 3) * kNSB * kNSB + threadIdx.x] = 0;
                for (int q = threadIdx.x, k = 0; q < kBT * kBT; q += blockDim.x, ++k) {
                    const int x = x0 + q % kBT, z = z0 + q / kBT;
                    if (x >= nx || z >= nz) continue;
                    const int bx = (q % kBT) / kSB, bz = (q / kBT) / kSB;
                    bool near = it == 0;
                    for (int dz = -1; dz <= 1 && !near; ++dz)
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int cx = bx + dx, cz = bz + dz;
                            if (cx >= 0 && cx < kNSB && cz >= 0 && cz < kNSB && prev[cz * kNSB + cx]) near = true;
                        }
                    if (!near) continue;
                    const int e = (q % kBT + H) + (q / kBT + H) * SW;
                    const T cur = wt[e];
                    const T best = pull(e, x, z, cur);
                    if (best < cur) {
                        wt[e] = best;
                        any = true;
                        changed |= 1u << k;
                        now[bz * kNSB + bx] = 1;
                    }
                }
                still = __syncthreads_or(any);
                if (!still) break;
            }
            for (int q = threadIdx.x, k = 0; q < kBT * kBT; q += blockDim.x, ++k) {   // write back, re-key
                const int lx = q % kBT, lz = q / kBT;
                const int x = x0 + lx, z = z0 + lz;
                if (x >= nx || z >= nz) continue;
                const T v = wt[(lx + H) + (lz + H) * SW];
                tau[(size_t)x + (size_t)nx * z] = v;
                if (!((changed >> k) & 1u)) continue;
                const Bits b = to_bits<T, Bits>(v);
                const int sx = lx < H ? 0 : lx >= kBT - H ? 2 : 1;          // side within reach in x
                const int sz = lz < H ? 0 : lz >= kBT - H ? 2 : 1;
                atomicMin(&m9[4], b);
                if (sx != 1) atomicMin(&m9[3 + sx], b);                     // block left or right
                if (sz != 1) atomicMin(&m9[sz * 3 + 1], b);                 // block above or below
                if (sx != 1 && sz != 1) atomicMin(&m9[sz * 3 + sx], b);     // diagonal block
            }
            __syncthreads();
            if (threadIdx.x < 9) {
                const T m = from_bits<T, Bits>(m9[threadIdx.x]);
                const int tx = kt % TX + (int)threadIdx.x % 3 - 1, tz = kt / TX + (int)threadIdx.x / 3 - 1;
                const bool self = threadIdx.x == 4;
                if (m < T(INFINITY) && tx >= 0 && tx < TX && tz >= 0 && tz < TZ && (!self || still)) {
                    T* kk = key + tz * TX + tx;
                    *kk = fmin(*kk, m);
                }
            }
            __syncthreads();
        }
        if (pops > max_pops) break;
        if (!verify_pass()) return swept + cycle + 1;
        for (int t = threadIdx.x; t < nt; t += blockDim.x) key[t] = T(0);   // rare: start over everywhere
        __syncthreads();
    }
    return -1;
}

// Shared memory of both kernels after their weight tables: key [nt], rv [32],
// window tau [SW*SW], window class [SW*SW] (if staged), ri [32], chg
// [3][kNSB^2], m9 [9] (8-byte aligned).
struct BhmTail {
    size_t key, rv, wt, wk, ri, chg, m9, end;
};
__host__ __device__ inline BhmTail bhm_tail(size_t at, int nt, int SW, size_t es, bool class_window) {
    BhmTail t;
    t.key = at;
    t.rv = t.key + (size_t)nt * es;
    t.wt = t.rv + 32 * es;
    t.wk = t.wt + (size_t)SW * SW * es;
    t.ri = t.wk + (class_window ? (size_t)SW * SW * 4 : 0);
    t.chg = t.ri + 32 * 4;
    t.m9 = (t.chg + 3 * kNSB * kNSB * 4 + 7) & ~size_t(7);
    t.end = t.m9 + 9 * 8;
    return t;
}

// swept > 0: the fields were swept for `swept` cycles first; the CTAs whose
// field converged there (status >= 0) return at once, the others solve their
// field again from the source.  (Continuing from the swept traveltimes was
// measured slower: fields that have not converged after a few cycles still
// have improvable nodes almost everywhere, and the blocks' keys then give a
// poor order.)
template <typename T, int WMODE>
__global__ void __launch_bounds__(1024) relax_bhm_kernel(FieldArgs a, Offsets off, int H, int swept) {
    if (swept > 0 && a.status[blockIdx.x] >= 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = a.n_classes;
    const int field = blockIdx.x >> 1;
    const int comp = blockIdx.x & 1;
    const int mode = field % a.n_modes;
    const int s = field / a.n_modes;
    const int nx = a.nx, nz = a.nz;
    const size_t n = static_cast<size_t>(nx) * nz;
    const int nt = ((nx + kBT - 1) / kBT) * ((nz + kBT - 1) / kBT);
    const int SW = kBT + 2 * H;

    Smem<T> sm;
    unsigned char* p = smem_raw;
    const size_t wcount = WMODE == 1 ? static_cast<size_t>(off.n) * nk * nk
                          : WMODE == 0 ? static_cast<size_t>(nk) * off.n : 0;
    sm.W = reinterpret_cast<T*>(p); p += wcount * sizeof(T);
    sm.L = reinterpret_cast<T*>(p); p += off.n * sizeof(T);
    int* ws = reinterpret_cast<int*>(p); p += off.n * 4;      // window shift of each offset
    sm.ring = nullptr;
    sm.cring = nullptr;
    sm.lists = nullptr;
    sm.counts = nullptr;
    const BhmTail tl = bhm_tail((size_t)(p - smem_raw + 15) & ~size_t(15), nt, SW, sizeof(T), true);
    T* wt = reinterpret_cast<T*>(smem_raw + tl.wt);
    int* wk = reinterpret_cast<int*>(smem_raw + tl.wk);

    const T* sel = static_cast<const T*>(comp == 0 ? a.Vsel : a.Asel) + static_cast<size_t>(mode) * nk * off.n;
    for (int o = threadIdx.x; o < off.n; o += blockDim.x) {
        const double ox = off.x[o], oz = off.z[o];
        sm.L[o] = T(a.dx * sqrt(ox * ox + oz * oz));
        ws[o] = off.x[o] + off.z[o] * SW;
    }
    __syncthreads();
    if (WMODE == 1) {
        for (int t = threadIdx.x; t < off.n * nk * nk; t += blockDim.x) {
            const int kj = t % nk, ki = (t / nk) % nk, o = t / (nk * nk);
            sm.W[t] = edge_w<T>(comp, sm.L[o], sel[ki * off.n + o], sel[kj * off.n + o]);
        }
    } else if (WMODE == 0) {
        for (int t = threadIdx.x; t < nk * off.n; t += blockDim.x) sm.W[t] = sel[t];
    }
    T* tau = static_cast<T*>(comp == 0 ? a.tauR : a.tauI) + static_cast<size_t>(field) * n;
    int32_t* par = comp == 0 ? a.parR : a.parI;
    if (par) par += static_cast<size_t>(field) * n;
    const int64_t src = a.src[s];
    const int used = bhm_field<T>(
        tau, nx, nz, src, a.max_cycles, swept, H, reinterpret_cast<T*>(smem_raw + tl.key),
        reinterpret_cast<T*>(smem_raw + tl.rv), reinterpret_cast<int*>(smem_raw + tl.ri), wt,
        reinterpret_cast<int*>(smem_raw + tl.chg), smem_raw + tl.m9,
        [&](int q, size_t g, bool in) { wk[q] = in ? clamp_class(a.cls[g], nk) : 0; },
        [&](int e, int, int, T cur) {
            const int kj = wk[e];
            T best = cur;
            for (int o = 0; o < off.n; ++o) {
                const T ti = wt[e - ws[o]];
                if (!(ti < best)) continue;
                best = fmin(best, ti + pull_weight<T, WMODE>(sm, sel, off.n, nk, comp, o, wk[e - ws[o]], kj));
            }
            return best;
        },
        [&]() { return verify<T, WMODE>(sm, sel, off, tau, a.cls, nx, nz, nk, comp, src, par); });
    if (threadIdx.x == 0) a.status[blockIdx.x] = used;
}

// The same block-heap marching on the standard stencil of radius R (the
// offsets of the specialised sweep kernel): the window shifts are compile-time
// immediates, and each pull reads its weight either from a class-pair table
// in shared memory in stencil order, W[(q*nk + k_i)*nk + k_j], or (PN) from
// the per-node weights that the sweeps computed, wrow[(mode*2+comp)][q][node].
// Weights, keys, order and results are those of relax_bhm_kernel.
struct BhmStd {
    short map[128];        // stencil index -> caller offset index
    const void* wrow;      // per-node weights (PN), row layout
};

template <typename T, int R, bool PN>
__global__ void __launch_bounds__(1024) relax_bhm_std_kernel(FieldArgs a, Offsets off, BhmStd b, int swept) {
    if (swept > 0 && a.status[blockIdx.x] >= 0) return;
    constexpr int N = fast::Stencil<R>::N;
    constexpr int SW = kBT + 2 * R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = a.n_classes;
    const int field = blockIdx.x >> 1;
    const int comp = blockIdx.x & 1;
    const int mode = field % a.n_modes;
    const int s = field / a.n_modes;
    const int nx = a.nx, nz = a.nz;
    const size_t n = static_cast<size_t>(nx) * nz;
    const int nt = ((nx + kBT - 1) / kBT) * ((nz + kBT - 1) / kBT);

    unsigned char* p = smem_raw;
    T* W = reinterpret_cast<T*>(p); p += PN ? 0 : (size_t)N * nk * nk * sizeof(T);
    T* Lc = reinterpret_cast<T*>(p); p += (size_t)off.n * sizeof(T);     // lengths, caller order
    const BhmTail tl = bhm_tail((size_t)(p - smem_raw + 15) & ~size_t(15), nt, SW, sizeof(T), !PN);
    T* wt = reinterpret_cast<T*>(smem_raw + tl.wt);
    int* wk = reinterpret_cast<int*>(smem_raw + tl.wk);      // class id * nk (class-pair table only)

    const T* sel = static_cast<const T*>(comp == 0 ? a.Vsel : a.Asel) + static_cast<size_t>(mode) * nk * off.n;
    for (int o = threadIdx.x; o < off.n; o += blockDim.x) {
        const double ox = off.x[o], oz = off.z[o];
        Lc[o] = T(a.dx * sqrt(ox * ox + oz * oz));
    }
    if constexpr (!PN) {
        for (int t = threadIdx.x; t < N * nk * nk; t += blockDim.x) {
            const int kj = t % nk, ki = (t / nk) % nk, q = t / (nk * nk);
            const int o = b.map[q];
            const double ox = off.x[o], oz = off.z[o];
            const T L = T(a.dx * sqrt(ox * ox + oz * oz));
            W[t] = edge_w<T>(comp, L, sel[ki * off.n + o], sel[kj * off.n + o]);
        }
    }
    const T* wrow = PN ? static_cast<const T*>(b.wrow) + (size_t)(mode * 2 + comp) * N * n : nullptr;
    T* tau = static_cast<T*>(comp == 0 ? a.tauR : a.tauI) + static_cast<size_t>(field) * n;
    int32_t* par = comp == 0 ? a.parR : a.parI;
    if (par) par += static_cast<size_t>(field) * n;
    const int64_t src = a.src[s];
    Smem<T> sm{};                                    // for the generic verification pass (global tables)
    sm.L = Lc;
    const int used = bhm_field<T>(
        tau, nx, nz, src, a.max_cycles, swept, R, reinterpret_cast<T*>(smem_raw + tl.key),
        reinterpret_cast<T*>(smem_raw + tl.rv), reinterpret_cast<int*>(smem_raw + tl.ri), wt,
        reinterpret_cast<int*>(smem_raw + tl.chg), smem_raw + tl.m9,
        [&](int q, size_t g, bool in) {
            if constexpr (!PN) wk[q] = in ? clamp_class(a.cls[g], nk) * nk : 0;
        },
        [&](int e, int x, int z, T cur) {
            T best = cur;
            if constexpr (PN) {
                const T* wj = wrow + (size_t)x + (size_t)nx * z;
                fast::static_for<N>([&](auto qc) {
                    constexpr int qq = decltype(qc)::value;
                    constexpr int sh = fast::Table<R>::v.x[qq] + fast::Table<R>::v.z[qq] * SW;
                    const T ti = wt[e - sh];
                    if (ti < best) best = fmin(best, ti + wj[(size_t)qq * n]);
                });
            } else {
                const T* Wj = W + wk[e] / nk;          // + q*nk*nk + k_i*nk
                fast::static_for<N>([&](auto qc) {
                    constexpr int qq = decltype(qc)::value;
                    constexpr int sh = fast::Table<R>::v.x[qq] + fast::Table<R>::v.z[qq] * SW;
                    const T ti = wt[e - sh];
                    if (ti < best) best = fmin(best, ti + Wj[qq * nk * nk + wk[e - sh]]);
                });
            }
            return best;
        },
        [&]() { return verify<T, 2>(sm, sel, off, tau, a.cls, nx, nz, nk, comp, src, par); });
    if (threadIdx.x == 0) a.status[blockIdx.x] = used;
}

// ------------------------------------------------------------ 3D relaxation
// A 3D lattice (node x + nx*(y + ny*z)) is relaxed by plane sweeps: a cycle
// runs the planes of constant z upward, of constant y and of constant x in
// both directions, and of constant z downward; in each, a node pulls from the
// offsets whose component along the sweep axis has the sweep's sign, i.e. from
// finished planes, so the nodes of one plane are independent.  A plane is
// processed in tiles of TU x TV nodes: the tile plus a halo of H nodes (H =
// the stencil's largest component) is staged from the planes behind into
// shared memory (tau and class), so each pull reads shared memory; tau itself
// lives in global memory.  A pull whose source tau_i is not below the current
// best is skipped without reading its class or weight (weights are >= 0, so
// it cannot improve).  The verification pass stages planes z-H..z+H and
// applies the 2D parent rule.
// 3D tile shapes (in-plane u x v nodes, one thread per node of a 512-thread
// CTA): 0 = 32 x 16 (the default), 1 = 64 x 8 (longer rows along x).
constexpr int kTU = 32, kTV = 16;

struct Stage3 {
    int H, SU, SV;      // halo, staged tile extents
};

// Several CTAs per field component ("parts", one cooperative launch, so all
// of them are resident): part p takes the tiles t = p, p + parts, ... of every
// plane, and the parts of a field meet at a barrier after each plane (a plane
// reads the planes behind it, tiles of the neighbours included).  Traveltimes
// other parts write are read through L2 (ld.cg), never from a stale L1 line.
constexpr int kSyncStride = 16;                 // unsigned words per field component (64 bytes)
constexpr long long kBarrierSpins = 1LL << 24;  // about a second of polling, then give up

struct Part3 {
    int part, parts;
    unsigned* word;         // this field component's barrier words, or null for one part
    unsigned gen;           // barriers passed so far
    bool failed;            // a barrier wait ran out (status -1, stop)
};

// Barrier of the parts of one field component; returns false (and marks the
// part failed) if the others did not all arrive within kBarrierSpins polls.
__device__ __forceinline__ bool part_barrier(Part3& pt) {
    if (pt.parts == 1) {
        __syncthreads();
        return true;
    }
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        __threadfence();
        atomicAdd(pt.word, 1u);
        const unsigned target = (pt.gen + 1) * (unsigned)pt.parts;
        long long spins = 0;
        while (*(volatile unsigned*)pt.word < target) {
            if (++spins > kBarrierSpins) { s_ok = 0; break; }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    ++pt.gen;
    if (!s_ok) pt.failed = true;
    return s_ok != 0;
}

template <typename TA>
__device__ __forceinline__ TA ld_tau(const TA* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ xf::ff ld_tau<xf::ff>(const xf::ff* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return xf::ff(v.x, v.y);
}

// In-plane coordinates (u, v) and plane p of a sweep along `axis` (0: x, 1: y,
// 2: z planes) -> node index.
__device__ __forceinline__ long long node3(int axis, int u, int v, int p, int nx, int ny) {
    if (axis == 2) return (long long)u + (long long)nx * ((long long)v + (long long)ny * p);
    if (axis == 1) return (long long)u + (long long)nx * ((long long)p + (long long)ny * v);
    return (long long)p + (long long)nx * ((long long)u + (long long)ny * v);
}

template <typename T>
__device__ __forceinline__ void stage_planes(T* st, int* sk, const T* tau, const int32_t* cls, int nk, int axis,
                                             int nu, int nv, int np, int p0, int pstep, int nplanes, int tu0,
                                             int tv0, const Stage3& g, int nx, int ny) {
    const int per = g.SU * g.SV;
    for (int e = threadIdx.x; e < nplanes * per; e += blockDim.x) {
        const int pl = p0 + pstep * (e / per);
        const int r = e % per;
        const int u = tu0 - g.H + r % g.SU, v = tv0 - g.H + r / g.SU;
        if (pl >= 0 && pl < np && u >= 0 && u < nu && v >= 0 && v < nv) {
            const long long j = node3(axis, u, v, pl, nx, ny);
            st[e] = ld_tau(tau + j);
            sk[e] = clamp_class(cls[j], nk);
        } else {
            st[e] = T(INFINITY);
            sk[e] = 0;
        }
    }
}

// TW: weight type; TA: traveltime accumulation and storage type (double,
// float, or float-float pairs for float weights with ~48-bit accumulation).
template <typename TW, typename TA, int WMODE, int TU, int TV>
__device__ bool sweep3d(const Smem<TW>& sm, const TW* __restrict__ gsel, const Offsets& off, const short* qo,
                        const short* qu, const short* qv, const short* ql, int cnt, int axis, int dir, TA* tau,
                        const int32_t* __restrict__ cls, int nx, int ny, int nz, int nk, int comp, TA* st, int* sk,
                        const Stage3& g, Part3& part) {
    const int nu = axis == 0 ? ny : nx;
    const int nv = axis == 2 ? ny : nz;
    const int np = axis == 2 ? nz : axis == 1 ? ny : nx;
    const int per = g.SU * g.SV;
    const int ntu = (nu + TU - 1) / TU;
    bool changed = false;
    for (int step = 0; step < np && !part.failed; ++step) {
        const int p = dir > 0 ? step : np - 1 - step;
        for (int tv0 = 0; tv0 < nv; tv0 += TV) {
            for (int tu0 = 0; tu0 < nu; tu0 += TU) {
                if (((tv0 / TV) * ntu + tu0 / TU) % part.parts != part.part) continue;
                // planes p - dir*1 .. p - dir*H at stage slots 0 .. H-1
                stage_planes(st, sk, tau, cls, nk, axis, nu, nv, np, p - dir, -dir, g.H, tu0, tv0, g, nx, ny);
                __syncthreads();
                const int u = tu0 + (int)(threadIdx.x % TU), v = tv0 + (int)(threadIdx.x / TU);
                if (threadIdx.x < TU * TV && u < nu && v < nv) {
                    const long long j = node3(axis, u, v, p, nx, ny);
                    const int kj = clamp_class(cls[j], nk);
                    const TA cur = ld_tau(tau + j);
                    TA best = cur;
                    const int su = u - tu0 + g.H, sv = v - tv0 + g.H;
                    for (int q = 0; q < cnt; ++q) {
                        const int e = (ql[q] - 1) * per + (sv - qv[q]) * g.SU + (su - qu[q]);
                        const TA ti = st[e];
                        if (!(ti < best)) continue;
                        best = fmin(best, ti + pull_weight<TW, WMODE>(sm, gsel, off.n, nk, comp, qo[q], sk[e], kj));
                    }
                    if (best < cur) {
                        tau[j] = best;
                        changed = true;
                    }
                }
                __syncthreads();
            }
        }
        part_barrier(part);                     // the plane is complete in every part
    }
    return __syncthreads_or(changed);
}

template <typename TW, typename TA, int WMODE, int TU, int TV>
__device__ bool verify3d(const Smem<TW>& sm, const TW* __restrict__ gsel, const Offsets& off, TA* tau,
                         const int32_t* __restrict__ cls, int nx, int ny, int nz, int nk, int comp, int64_t src,
                         int32_t* par, TA* st, int* sk, const Stage3& g, Part3& part) {
    const int per = g.SU * g.SV;
    const int ntx = (nx + TU - 1) / TU;
    bool changed = false;
    for (int z = 0; z < nz && !part.failed; ++z) {
        for (int ty0 = 0; ty0 < ny; ty0 += TV) {
            for (int tx0 = 0; tx0 < nx; tx0 += TU) {
                if (((ty0 / TV) * ntx + tx0 / TU) % part.parts != part.part) continue;
                // planes z-H .. z+H at stage slots 0 .. 2H
                stage_planes(st, sk, tau, cls, nk, 2, nx, ny, nz, z - g.H, 1, 2 * g.H + 1, tx0, ty0, g, nx, ny);
                __syncthreads();
                const int x = tx0 + (int)(threadIdx.x % TU), y = ty0 + (int)(threadIdx.x / TU);
                if (threadIdx.x < TU * TV && x < nx && y < ny) {
                    const long long j = node3(2, x, y, z, nx, ny);
                    const int kj = clamp_class(cls[j], nk);
                    const TA cur = ld_tau(tau + j);
                    TA best = TA(INFINITY);
                    long long bi = -1;
                    const int sx = x - tx0 + g.H, sy = y - ty0 + g.H;
                    for (int o = 0; o < off.n; ++o) {
                        const int xi = x - off.x[o], yi = y - off.y[o], zi = z - off.z[o];
                        if (xi < 0 || xi >= nx || yi < 0 || yi >= ny || zi < 0 || zi >= nz) continue;
                        const int e = (g.H - off.z[o]) * per + (sy - off.y[o]) * g.SU + (sx - off.x[o]);
                        const TA ti = st[e];
                        if (ti > best) continue;
                        const TA c = ti + pull_weight<TW, WMODE>(sm, gsel, off.n, nk, comp, o, sk[e], kj);
                        const long long i = node3(2, xi, yi, zi, nx, ny);
                        if (c < best || (c == best && i < bi)) { best = c; bi = i; }
                    }
                    if (best < cur) {
                        tau[j] = best;
                        changed = true;
                    } else if (par) {
                        par[j] = (j == src) ? static_cast<int32_t>(src) : (!(cur < TA(INFINITY)) ? -1 : (int32_t)bi);
                    }
                }
                __syncthreads();
            }
        }
        part_barrier(part);
    }
    return __syncthreads_or(changed);
}

// ---- the standard 3D stencil of reach 2, unrolled
// The 98 lattice directions (ox, oy, oz) with max(|ox|, |oy|, |oz|) <= 2 and
// gcd(|ox|, |oy|, |oz|) = 1 (the 26 neighbours and 72 secondary nodes), in
// the order of the callers' offset arrays: oz, then oy, then ox ascending.
// When a launch's offsets are exactly this table and the class-pair weight
// table is in shared memory, the sweeps and the verification unroll the
// stencil at compile time: a pull's stage index is the thread's base plus a
// constant and its weight index a constant plus the class pair, where the
// general form loads four list entries and recomputes both per pull.  Same
// pulls, same comparisons: the fields and parents are those of the general
// form, bit for bit.
struct Stencil3 {
    static constexpr int N = 98;
    int x[N], y[N], z[N];
    constexpr Stencil3() : x(), y(), z() {
        int n = 0;
        for (int zz = -2; zz <= 2; ++zz)
            for (int yy = -2; yy <= 2; ++yy)
                for (int xx = -2; xx <= 2; ++xx)
                    if ((xx || yy || zz) &&
                        fast::cgcd(fast::cgcd(fast::cabs(xx), fast::cabs(yy)), fast::cabs(zz)) == 1 && n < N) {
                        x[n] = xx; y[n] = yy; z[n] = zz; ++n;
                    }
    }
};
constexpr int stencil3_count() {
    int n = 0;
    for (int zz = -2; zz <= 2; ++zz)
        for (int yy = -2; yy <= 2; ++yy)
            for (int xx = -2; xx <= 2; ++xx)
                n += (xx || yy || zz) && fast::cgcd(fast::cgcd(fast::cabs(xx), fast::cabs(yy)), fast::cabs(zz)) == 1;
    return n;
}
static_assert(stencil3_count() == Stencil3::N, "the reach-2 3D stencil has 98 directions");
template <int D>
struct Table3 {
    static constexpr Stencil3 v{};
};
// Pulls between compiler fences in the unrolled loops (register pressure:
// without fences every stage load of a sweep is hoisted ahead of the first
// pull, and the kernel needs 128 registers, one CTA per SM).
constexpr int kFence3 = 6;

// Float-float traveltimes (float weights): a candidate ti + w whose float sum
// fl(ti.hi + w) is above best.hi * (1 + 2^-21) exceeds best exactly (the
// dropped ti.lo and the two roundings move it by under 3 * 2^-24 relative;
// ti, w >= 0), so the float-float addition and comparison are skipped for it.
// The skipped candidates would lose anyway, ties included (at best = 0 the
// test is fl(ti.hi + w) > 0, which no tie at 0 passes): same results, fewer
// instructions.
__device__ __forceinline__ float ff_skip_above(const xf::ff& best) { return best.hi * (1.0f + 0x1p-21f); }

// sweep3d over the unrolled stencil: sweep along AXIS (0: x, 1: y, 2: z
// planes) in direction DIR; halo H = 2; weights from the class-pair table
// W[o][k_i][k_j].
template <typename TW, typename TA, int TU, int TV, int AXIS, int DIR>
__device__ bool sweep3d_std(const Smem<TW>& sm, TA* tau, const int32_t* __restrict__ cls, int nx, int ny, int nz,
                            int nk, TA* st, int* sk, Part3& part) {
    constexpr int H = 2, SU = TU + 2 * H, SV = TV + 2 * H, per = SU * SV;
    constexpr bool kFF = std::is_same<TA, xf::ff>::value;
    const Stage3 g{H, SU, SV};
    const int nu = AXIS == 0 ? ny : nx;
    const int nv = AXIS == 2 ? ny : nz;
    const int np = AXIS == 2 ? nz : AXIS == 1 ? ny : nx;
    const int ntu = (nu + TU - 1) / TU;
    const int nk2 = nk * nk;
    bool changed = false;
    for (int step = 0; step < np && !part.failed; ++step) {
        const int p = DIR > 0 ? step : np - 1 - step;
        for (int tv0 = 0; tv0 < nv; tv0 += TV) {
            for (int tu0 = 0; tu0 < nu; tu0 += TU) {
                if (((tv0 / TV) * ntu + tu0 / TU) % part.parts != part.part) continue;
                // planes p - DIR*1 .. p - DIR*H at stage slots 0 .. H-1
                stage_planes(st, sk, tau, cls, nk, AXIS, nu, nv, np, p - DIR, -DIR, H, tu0, tv0, g, nx, ny);
                __syncthreads();
                const int u = tu0 + (int)(threadIdx.x % TU), v = tv0 + (int)(threadIdx.x / TU);
                if (threadIdx.x < TU * TV && u < nu && v < nv) {
                    const long long j = node3(AXIS, u, v, p, nx, ny);
                    const int kj = clamp_class(cls[j], nk);
                    const TA cur = ld_tau(tau + j);
                    TA best = cur;
                    const int base = (v - tv0 + H) * SU + (u - tu0 + H);
                    const TW* Wj = sm.W + kj;
                    [[maybe_unused]] float skip = 0.0f;
                    if constexpr (kFF) skip = ff_skip_above(best);
                    fast::static_for<Stencil3::N>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        constexpr int ox = Table3<0>::v.x[q], oy = Table3<0>::v.y[q], oz = Table3<0>::v.z[q];
                        constexpr int oa = AXIS == 2 ? oz : AXIS == 1 ? oy : ox;
                        if constexpr (oa * DIR > 0) {
                            constexpr int ou = AXIS == 0 ? oy : ox;
                            constexpr int ov = AXIS == 2 ? oy : oz;
                            constexpr int d = (oa * DIR - 1) * per - ov * SU - ou;
                            const TA ti = st[base + d];
                            if (ti < best) {
                                const TW w = Wj[q * nk2 + sk[base + d] * nk];
                                if constexpr (kFF) {
                                    if (ti.hi + w <= skip) {
                                        best = fmin(best, ti + w);
                                        skip = ff_skip_above(best);
                                    }
                                } else {
                                    best = fmin(best, ti + w);
                                }
                            }
                            // a compiler fence every kFence3 entries keeps the
                            // loads of a few pulls in flight, not of all of them
                            if constexpr (q % kFence3 == kFence3 - 1) asm volatile("" ::: "memory");
                        }
                    });
                    if (best < cur) {
                        tau[j] = best;
                        changed = true;
                    }
                }
                __syncthreads();
            }
        }
        part_barrier(part);                     // the plane is complete in every part
    }
    return __syncthreads_or(changed);
}

// verify3d over the unrolled stencil (in-neighbours in offset order, the
// parent rule's tie break on the smaller node index as in verify3d).
template <typename TW, typename TA, int TU, int TV>
__device__ bool verify3d_std(const Smem<TW>& sm, TA* tau, const int32_t* __restrict__ cls, int nx, int ny, int nz,
                             int nk, int64_t src, int32_t* par, TA* st, int* sk, Part3& part) {
    constexpr int H = 2, SU = TU + 2 * H, SV = TV + 2 * H, per = SU * SV;
    constexpr bool kFF = std::is_same<TA, xf::ff>::value;
    const Stage3 g{H, SU, SV};
    const int ntx = (nx + TU - 1) / TU;
    const int nk2 = nk * nk;
    bool changed = false;
    for (int z = 0; z < nz && !part.failed; ++z) {
        for (int ty0 = 0; ty0 < ny; ty0 += TV) {
            for (int tx0 = 0; tx0 < nx; tx0 += TU) {
                if (((ty0 / TV) * ntx + tx0 / TU) % part.parts != part.part) continue;
                // planes z-H .. z+H at stage slots 0 .. 2H
                stage_planes(st, sk, tau, cls, nk, 2, nx, ny, nz, z - H, 1, 2 * H + 1, tx0, ty0, g, nx, ny);
                __syncthreads();
                const int x = tx0 + (int)(threadIdx.x % TU), y = ty0 + (int)(threadIdx.x / TU);
                if (threadIdx.x < TU * TV && x < nx && y < ny) {
                    const long long j = node3(2, x, y, z, nx, ny);
                    const int kj = clamp_class(cls[j], nk);
                    const TA cur = ld_tau(tau + j);
                    TA best = TA(INFINITY);
                    long long bi = -1;
                    const int base = H * per + (y - ty0 + H) * SU + (x - tx0 + H);
                    const TW* Wj = sm.W + kj;
                    [[maybe_unused]] float skip = INFINITY;
                    fast::static_for<Stencil3::N>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        constexpr int ox = Table3<0>::v.x[q], oy = Table3<0>::v.y[q], oz = Table3<0>::v.z[q];
                        constexpr int d = -oz * per - oy * SU - ox;
                        const int xi = x - ox, yi = y - oy, zi = z - oz;
                        if (xi >= 0 && xi < nx && yi >= 0 && yi < ny && zi >= 0 && zi < nz) {
                            const TA ti = st[base + d];
                            if (!(ti > best)) {
                                const TW w = Wj[q * nk2 + sk[base + d] * nk];
                                bool take = true;
                                if constexpr (kFF) take = ti.hi + w <= skip;
                                if (take) {
                                    const TA c = ti + w;
                                    const long long i = node3(2, xi, yi, zi, nx, ny);
                                    if (c < best || (c == best && i < bi)) {
                                        best = c;
                                        bi = i;
                                        if constexpr (kFF) skip = ff_skip_above(best);
                                    }
                                }
                            }
                        }
                        if constexpr (q % kFence3 == kFence3 - 1) asm volatile("" ::: "memory");
                    });
                    if (best < cur) {
                        tau[j] = best;
                        changed = true;
                    } else if (par) {
                        par[j] = (j == src) ? static_cast<int32_t>(src) : (!(cur < TA(INFINITY)) ? -1 : (int32_t)bi);
                    }
                }
                __syncthreads();
            }
        }
        part_barrier(part);
    }
    return __syncthreads_or(changed);
}

// Shared memory of relax3d_kernel after the weight table: L [n_off], six
// per-sweep lists of (offset, in-plane u, in-plane v, lag) as shorts, counts,
// then the stage (tau, then class) for 2H+1 planes.
__host__ __device__ inline size_t stage3_elems(int H, int TU = kTU, int TV = kTV) {
    return (size_t)(2 * H + 1) * (TU + 2 * H) * (TV + 2 * H);
}

// TA = xf::ff: float weights, traveltimes accumulated as float-float pairs in
// the (double) output arrays, converted to double in place at the end.
// One field component fc (= field * 2 + component) of one lattice, by the
// CTA (or, parts > 1, by part `part_idx` of a cooperative group of CTAs).
template <typename T, typename TA, int WMODE, int TU, int TV>
__device__ void relax3d_field(const FieldArgs& a, const Offsets& off, int H, int fc, int part_idx,
                              unsigned char* smem_raw) {
    const int nk = a.n_classes;
    const int field = fc >> 1;
    const int comp = fc & 1;
    Part3 part{part_idx, a.parts, a.parts > 1 ? a.sync + (size_t)fc * kSyncStride : nullptr, 0u, false};
    const int mode = field % a.n_modes;
    const int s = field / a.n_modes;
    const size_t n = (size_t)a.nx * a.ny * a.nz;

    Smem<T> sm;
    unsigned char* p = smem_raw;
    const size_t wcount = WMODE == 1 ? static_cast<size_t>(off.n) * nk * nk
                          : WMODE == 0 ? static_cast<size_t>(nk) * off.n : 0;
    sm.W = reinterpret_cast<T*>(p); p += wcount * sizeof(T);
    sm.L = reinterpret_cast<T*>(p); p += off.n * sizeof(T);
    Stage3 g{H, TU + 2 * H, TV + 2 * H};
    TA* st = reinterpret_cast<TA*>(p); p += stage3_elems(H, TU, TV) * sizeof(TA);
    int* sk = reinterpret_cast<int*>(p); p += stage3_elems(H, TU, TV) * sizeof(int);
    sm.ring = nullptr;
    sm.cring = nullptr;
    short* lists = reinterpret_cast<short*>(p); p += 4 * 6 * off.n * sizeof(short);
    sm.lists = lists;
    sm.counts = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(p) + 3) & ~uintptr_t(3));

    const T* sel = static_cast<const T*>(comp == 0 ? a.Vsel : a.Asel) + static_cast<size_t>(mode) * nk * off.n;
    for (int o = threadIdx.x; o < off.n; o += blockDim.x) {
        const double ox = off.x[o], oy = off.y[o], oz = off.z[o];
        sm.L[o] = T(a.dx * sqrt(ox * ox + oy * oy + oz * oz));
    }
    __syncthreads();
    if (WMODE == 1) {
        for (int t = threadIdx.x; t < off.n * nk * nk; t += blockDim.x) {
            const int kj = t % nk, ki = (t / nk) % nk, o = t / (nk * nk);
            sm.W[t] = edge_w<T>(comp, sm.L[o], sel[ki * off.n + o], sel[kj * off.n + o]);
        }
    } else if (WMODE == 0) {
        for (int t = threadIdx.x; t < nk * off.n; t += blockDim.x) sm.W[t] = sel[t];
    }
    // list l of sweep (axis, dir): 0 (z,+) 1 (y,+) 2 (x,+) 3 (x,-) 4 (y,-) 5 (z,-);
    // entries: offset index, in-plane components (u, v) and lag along the axis
    const int ax[6] = {2, 1, 0, 0, 1, 2}, dr[6] = {1, 1, 1, -1, -1, -1};
    if (threadIdx.x < 6) {
        const int l = threadIdx.x, axis = ax[l], dir = dr[l];
        short* qo = lists + (4 * l + 0) * off.n;
        short* qu = lists + (4 * l + 1) * off.n;
        short* qv = lists + (4 * l + 2) * off.n;
        short* ql = lists + (4 * l + 3) * off.n;
        int c = 0;
        for (int o = 0; o < off.n; ++o) {
            const int oa = axis == 2 ? off.z[o] : axis == 1 ? off.y[o] : off.x[o];
            if (oa * dir <= 0) continue;
            qo[c] = (short)o;
            qu[c] = axis == 0 ? off.y[o] : off.x[o];
            qv[c] = axis == 2 ? off.y[o] : off.z[o];
            ql[c] = (short)(oa * dir);
            ++c;
        }
        sm.counts[l] = c;
    }

    TA* tau = static_cast<TA*>(comp == 0 ? a.tauR : a.tauI) + static_cast<size_t>(field) * n;
    int32_t* par = comp == 0 ? a.parR : a.parI;
    if (par) par += static_cast<size_t>(field) * n;
    const int64_t src = a.src[s];
    const size_t stride = (size_t)blockDim.x * part.parts;
    for (size_t j = threadIdx.x + (size_t)part.part * blockDim.x; j < n; j += stride)
        tau[j] = (j == (size_t)src) ? TA(0.0f) : TA(INFINITY);
    part_barrier(part);

    int used = -1;
    const bool unrolled = WMODE == 1 && a.std3 && H == 2;
    for (int cycle = 0; cycle < a.max_cycles && !part.failed; ++cycle) {
        bool changed;
        if (WMODE == 1 && unrolled) {
            // the six sweeps in the general form's order: (z,+) (y,+) (x,+) (x,-) (y,-) (z,-)
            sweep3d_std<T, TA, TU, TV, 2, 1>(sm, tau, a.cls, a.nx, a.ny, a.nz, nk, st, sk, part);
            sweep3d_std<T, TA, TU, TV, 1, 1>(sm, tau, a.cls, a.nx, a.ny, a.nz, nk, st, sk, part);
            sweep3d_std<T, TA, TU, TV, 0, 1>(sm, tau, a.cls, a.nx, a.ny, a.nz, nk, st, sk, part);
            sweep3d_std<T, TA, TU, TV, 0, -1>(sm, tau, a.cls, a.nx, a.ny, a.nz, nk, st, sk, part);
            sweep3d_std<T, TA, TU, TV, 1, -1>(sm, tau, a.cls, a.nx, a.ny, a.nz, nk, st, sk, part);
            sweep3d_std<T, TA, TU, TV, 2, -1>(sm, tau, a.cls, a.nx, a.ny, a.nz, nk, st, sk, part);
            changed = verify3d_std<T, TA, TU, TV>(sm, tau, a.cls, a.nx, a.ny, a.nz, nk, src, par, st, sk, part);
        } else {
            for (int l = 0; l < 6; ++l)
                sweep3d<T, TA, WMODE, TU, TV>(sm, sel, off, lists + (4 * l) * off.n, lists + (4 * l + 1) * off.n,
                                  lists + (4 * l + 2) * off.n, lists + (4 * l + 3) * off.n, sm.counts[l], ax[l],
                                  dr[l], tau, a.cls, a.nx, a.ny, a.nz, nk, comp, st, sk, g, part);
            changed = verify3d<T, TA, WMODE, TU, TV>(sm, sel, off, tau, a.cls, a.nx, a.ny, a.nz, nk, comp, src, par,
                                                     st, sk, g, part);
        }
        if (part.parts > 1) {
            // OR of the parts' verdicts in flag word 1 + (cycle & 1); the other
            // flag word, last read a cycle ago, is cleared for the next cycle
            unsigned* flag = part.word + 1 + (cycle & 1);
            if (threadIdx.x == 0 && changed) atomicOr(flag, 1u);
            part_barrier(part);
            changed = *(volatile unsigned*)flag != 0;
            if (threadIdx.x == 0 && part.part == 0) part.word[1 + ((cycle + 1) & 1)] = 0u;
        }
        if (part.failed) break;
        if (!changed) {
            used = cycle + 1;
            break;
        }
    }
    if constexpr (std::is_same<TA, xf::ff>::value) {
        part_barrier(part);
        double* out = reinterpret_cast<double*>(tau);          // same 8 bytes per node
        for (size_t j = threadIdx.x + (size_t)part.part * blockDim.x; j < n; j += stride) {
            const xf::ff v = ld_tau(tau + j);
            out[j] = double(v.hi) + double(v.lo);
        }
    }
    if (threadIdx.x == 0 && part.part == 0) a.status[fc] = part.failed ? -1 : used;
}

template <typename T, typename TA, int WMODE, int TU, int TV>
__global__ void __launch_bounds__(512, 2) relax3d_kernel(FieldArgs a, Offsets off, int H) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    relax3d_field<T, TA, WMODE, TU, TV>(a, off, H, (int)(blockIdx.x / a.parts), (int)(blockIdx.x % a.parts),
                                        smem_raw);
}

// Several 3D lattices in one persistent launch: the work items are the field
// components of every lattice, numbered lattice by lattice (start[l] .. 
// start[l + 1] - 1; the host orders the lattices largest first, so that the
// longest items start first).  Each CTA claims the next item from a device
// counter (zeroed before the launch) until none is left, and relaxes it with
// the lattice's own arguments from the table (a kernel parameter, read in
// place).  One CTA per item: parts = 1 in every entry.
constexpr int kMaxLattices = 48;

struct LatticeTable {
    int n;
    long long start[kMaxLattices + 1];
    FieldArgs a[kMaxLattices];
};

template <typename T, typename TA, int WMODE, int TU, int TV>
__global__ void __launch_bounds__(512, 2) relax3d_multi_kernel(const __grid_constant__ LatticeTable t,
                                                            const __grid_constant__ Offsets off, int H,
                                                            unsigned long long* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_item;
    const long long total = t.start[t.n];
    for (;;) {
        __syncthreads();                      // the previous item's shared memory is no longer read
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        int l = 0;
        while (l + 1 < t.n && t.start[l + 1] <= item) ++l;
        relax3d_field<T, TA, WMODE, TU, TV>(t.a[l], off, H, (int)(item - t.start[l]), 0, smem_raw);
    }
}

// ------------------------------------------------------------ parent ties
// Tie log of the parent rule (Eq. 33): node j of a converged field is a tie
// when its second-best in-neighbour candidate tau_i + w_ij lies within
// rel_tol * best of the best one, i.e. when rounding at that level can pick
// either predecessor.  The weights are those of the relaxation (same lookup
// tables and rounding, Eq. 28-30); candidates are formed in the traveltime
// type TT.  One thread per node; blockIdx.y = field, blockIdx.z = component.
template <typename TW, typename TT>
__global__ void parent_ties_kernel(const TW* __restrict__ Vsel, const TW* __restrict__ Asel, int n_modes, int nk,
                                   Offsets off, int nx, int ny, int nz, double dx,
                                   const int32_t* __restrict__ cls, const int64_t* __restrict__ src,
                                   const TT* __restrict__ tauR, const TT* __restrict__ tauI, double rel_tol,
                                   uint8_t* __restrict__ tieR, uint8_t* __restrict__ tieI,
                                   unsigned long long* __restrict__ counts) {
    __shared__ TW L[kMaxOff];
    __shared__ int block_ties;
    for (int o = threadIdx.x; o < off.n; o += blockDim.x) {
        const double ox = off.x[o], oy = off.y[o], oz = off.z[o];
        L[o] = TW(dx * sqrt(ox * ox + oy * oy + oz * oz));
    }
    if (threadIdx.x == 0) block_ties = 0;
    __syncthreads();
    const int field = blockIdx.y, comp = blockIdx.z;
    const int mode = field % n_modes;
    const size_t n = (size_t)nx * ny * nz;
    const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool tie = false;
    if (j < n) {
        const TT* tau = (comp == 0 ? tauR : tauI) + (size_t)field * n;
        const TW* sel = (comp == 0 ? Vsel : Asel) + (size_t)mode * nk * off.n;
        const int64_t s = src[field / n_modes];
        if ((int64_t)j != s && !isinf(tau[j])) {
            const int xj = (int)(j % nx), yj = (int)((j / nx) % ny), zj = (int)(j / ((size_t)nx * ny));
            const int kj = clamp_class(cls[j], nk);
            TT best = TT(INFINITY), second = TT(INFINITY);
            for (int o = 0; o < off.n; ++o) {
                const int xi = xj - off.x[o], yi = yj - off.y[o], zi = zj - off.z[o];
                if (xi < 0 || xi >= nx || yi < 0 || yi >= ny || zi < 0 || zi >= nz) continue;
                const size_t i = (size_t)xi + (size_t)nx * ((size_t)yi + (size_t)ny * zi);
                const int ki = clamp_class(cls[i], nk);
                const TW w = edge_w<TW>(comp, L[o], sel[(size_t)ki * off.n + o], sel[(size_t)kj * off.n + o]);
                const TT c = tau[i] + TT(w);
                if (c < best) { second = best; best = c; }
                else if (c < second) second = c;
            }
            tie = !isinf(second) && double(second) - double(best) <= rel_tol * double(best);
        }
        uint8_t* out = comp == 0 ? tieR : tieI;
        if (out) out[(size_t)field * n + j] = tie ? 1 : 0;
    }
    if (tie) atomicAdd(&block_ties, 1);
    __syncthreads();
    if (threadIdx.x == 0 && counts && block_ties) atomicAdd(counts + field * 2 + comp, (unsigned long long)block_ties);
}

// ------------------------------------------------------------ raypaths
// One thread per (field, receiver): walk the parents once to count the path
// (bounded by cap), then again to write it source-first.
__global__ void raypath_kernel(const int32_t* __restrict__ par, int n_fields, int64_t n_nodes,
                               const int64_t* __restrict__ src, const int64_t* __restrict__ rcv,
                               int n_rcv, int64_t cap, int64_t* __restrict__ paths,
                               int64_t* __restrict__ len) {
    const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<long long>(n_fields) * n_rcv) return;
    const int f = static_cast<int>(t / n_rcv);
    const int32_t* p = par + static_cast<size_t>(f) * n_nodes;
    const int64_t s = src[f];
    int64_t node = rcv[t % n_rcv];
    int64_t count = 0;
    bool ok = node >= 0 && node < n_nodes;
    while (ok) {
        ++count;
        if (node == s) break;
        if (count >= cap) { ok = false; break; }
        const int64_t nxt = p[node];
        if (nxt < 0 || nxt >= n_nodes) { ok = false; break; }
        node = nxt;
    }
    if (!ok) { len[t] = 0; return; }
    len[t] = count;
    node = rcv[t % n_rcv];
    int64_t* out = paths + static_cast<size_t>(t) * cap;
    for (int64_t q = count - 1; q >= 0; --q) {
        out[q] = node;
        if (q > 0) node = p[node];
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct WsLayout {
    size_t sel, idx, src, status, rowk, sync, total;
};

constexpr int kRowkMax = 2048;       // rows of a 2D lattice the row-class path handles

WsLayout ws_layout(int n_modes, int n_classes, int n_off, int precision, int n_sources) {
    const size_t es = precision == CHERT_FP64 ? 8 : 4;
    const size_t m = static_cast<size_t>(n_modes) * n_classes * n_off;
    WsLayout w;
    w.sel = 0;
    w.idx = align256(2 * m * es);
    w.src = w.idx + align256(m * 4);
    w.status = w.src + align256(static_cast<size_t>(n_sources) * 8);
    w.rowk = w.status + align256((static_cast<size_t>(n_sources) * n_modes * 2 + 1) * 4);
    w.sync = w.rowk + align256(static_cast<size_t>(kRowkMax) * 4);
    w.total = w.sync + align256(static_cast<size_t>(n_sources) * n_modes * 2 * kSyncStride * 4);
    return w;
}

int fill_offsets(Offsets& o, const int32_t* offsets, int n_off, const char* who) {
    CHERT_REQUIRE(offsets != nullptr, "%s: offsets is NULL", who);
    CHERT_REQUIRE(n_off >= 1 && n_off <= kMaxOff, "%s: n_off=%d (1..%d)", who, n_off, kMaxOff);
    o.n = n_off;
    for (int i = 0; i < n_off; i++) {
        const int32_t x = offsets[3 * i], y = offsets[3 * i + 1], z = offsets[3 * i + 2];
        CHERT_REQUIRE(x || y || z, "%s: zero offset", who);
        CHERT_REQUIRE(abs(x) < 32768 && abs(y) < 32768 && abs(z) < 32768, "%s: offset too large", who);
        o.x[i] = (short)x; o.y[i] = (short)y; o.z[i] = (short)z;
    }
    return CHERT_OK;
}

}  // namespace
}  // namespace chert

using namespace chert;

extern "C" int chert_edge_table(const chert_cache_arrays* cache, int n_modes, int n_classes,
                                int n_dir, int precision, const int32_t* offsets, int n_off,
                                int32_t* d_idx, void* d_Vsel, void* d_Asel, void* stream) {
    CHERT_REQUIRE(cache && cache->V && cache->A && cache->rx && cache->rz && cache->flag,
                  "chert_edge_table: cache arrays V, A, rx, rz, flag are required");
    CHERT_REQUIRE(d_idx && d_Vsel && d_Asel, "chert_edge_table: NULL output");
    CHERT_REQUIRE(n_modes >= 1 && n_classes >= 1 && n_dir >= 1, "chert_edge_table: bad counts");
    Offsets off;
    int rc = fill_offsets(off, offsets, n_off, "chert_edge_table");
    if (rc) return rc;
    const long long warps = static_cast<long long>(n_modes) * n_classes * n_off;
    const unsigned blocks = static_cast<unsigned>((warps * 32 + 255) / 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == CHERT_FP64) {
        edge_table_kernel<double><<<blocks, 256, 0, s>>>(
            (const double*)cache->rx, (const double*)cache->ry, (const double*)cache->rz, (const double*)cache->V,
            (const double*)cache->A, cache->flag, n_modes, n_classes, n_dir, off, d_idx,
            (double*)d_Vsel, (double*)d_Asel);
    } else {
        CHERT_REQUIRE(precision == CHERT_FP32 || precision == CHERT_MIXED,
                      "chert_edge_table: precision=%d", precision);
        edge_table_kernel<float><<<blocks, 256, 0, s>>>(
            (const float*)cache->rx, (const float*)cache->ry, (const float*)cache->rz, (const float*)cache->V,
            (const float*)cache->A, cache->flag, n_modes, n_classes, n_dir, off, d_idx,
            (float*)d_Vsel, (float*)d_Asel);
    }
    return launch_check("chert_edge_table");
}


// 3D launch: one CTA per field component, or, when the field components
// leave SMs idle, `parts` CTAs each (at most 8, every CTA of the grid
// resident: a cooperative launch), sharing each plane's tiles.  Under stream
// capture, one CTA per field component.
template <typename T, int WMODE, typename TA, int TU, int TV>
static int launch_relax3d(FieldArgs a, const Offsets& off, int H, size_t smem, int blocks, cudaStream_t s) {
    auto kern = relax3d_kernel<T, TA, WMODE, TU, TV>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime: smem attribute");
    int parts = 1;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime: capture status");
    int dev = 0, n_sm = 0, coop = 0, per_sm = 0;
    if (cap == cudaStreamCaptureStatusNone && a.sync && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, smem) == cudaSuccess && per_sm > 0) {
        const long long slots = (long long)per_sm * n_sm;
        const int tiles = std::min({((a.nx + TU - 1) / TU) * ((a.ny + TV - 1) / TV),
                                    ((a.nx + TU - 1) / TU) * ((a.nz + TV - 1) / TV),
                                    ((a.ny + TU - 1) / TU) * ((a.nz + TV - 1) / TV)});
        parts = (int)std::max(1LL, std::min<long long>({8LL, slots / blocks, (long long)tiles}));
    }
    cudaGetLastError();
    a.parts = parts;
    if (parts == 1) {
        kern<<<blocks, 512, smem, s>>>(a, off, H);
        return launch_check("chert_traveltime: relax3d");
    }
    e = cudaMemsetAsync(a.sync, 0, sizeof(unsigned) * (size_t)blocks * kSyncStride, s);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime: relax3d barrier words");
    void* args[] = {&a, const_cast<Offsets*>(&off), &H};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks * parts), dim3(512), args, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime: relax3d (cooperative)");
    return launch_check("chert_traveltime: relax3d");
}

template <typename T, int WMODE>
static int launch_bhm(const FieldArgs& a, const Offsets& off, int H, int swept, size_t smem, int blocks,
                      cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(relax_bhm_kernel<T, WMODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime: smem attribute");
    relax_bhm_kernel<T, WMODE><<<blocks, 1024, smem, s>>>(a, off, H, swept);
    return launch_check("chert_traveltime: block heap");
}

template <typename T, int WMODE>
static int launch_relax(const FieldArgs& a, const Offsets& off, size_t smem, int blocks,
                        cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(relax_kernel<T, WMODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime: smem attribute");
    relax_kernel<T, WMODE><<<blocks, 512, smem, s>>>(a, off);
    return launch_check("chert_traveltime: relax");
}

// ---- dispatch to the kernel specialised for the standard stencil ----------
// If the caller's offsets are exactly the standard radius-R stencil (in any
// order), map[q] receives the caller's index of stencil entry q.
template <int R>
static bool standard_map(const Offsets& off, short* map) {
    constexpr fast::Stencil<R> st{};
    if (off.n != fast::Stencil<R>::N) return false;
    for (int q = 0; q < fast::Stencil<R>::N; ++q) {
        int found = -1;
        for (int i = 0; i < off.n; ++i)
            if (off.x[i] == st.x[q] && off.z[i] == st.z[q] && off.y[i] == 0) { found = i; break; }
        if (found < 0) return false;
        map[q] = (short)found;
    }
    return true;
}

template <typename T, int R, bool PN>
static int launch_bhm_std(const FieldArgs& a, const Offsets& off, const BhmStd& b, int swept, size_t smem,
                          int blocks, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(relax_bhm_std_kernel<T, R, PN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime: smem attribute");
    relax_bhm_std_kernel<T, R, PN><<<blocks, 1024, smem, s>>>(a, off, b, swept);
    return launch_check("chert_traveltime: block heap");
}

// Block-heap marching on the standard stencil of radius R, if the offsets are
// that stencil and its tables fit: 1 launched, 0 not applicable, < 0 error.
// wrow: the per-node weights of the sweeps, or null (class-pair table).
template <typename T, int R>
static int try_bhm_std_R(const FieldArgs& a, const Offsets& off, const void* wrow, int swept, int smem_max,
                         int blocks, cudaStream_t s) {
    BhmStd b;
    if (!standard_map<R>(off, b.map)) return 0;
    b.wrow = wrow;
    constexpr int N = fast::Stencil<R>::N;
    const size_t es = sizeof(T);
    const size_t nt = (size_t)((a.nx + kBT - 1) / kBT) * ((a.nz + kBT - 1) / kBT);
    int rc;
    if (wrow) {
        const size_t smem = bhm_tail(((size_t)off.n * es + 15) & ~size_t(15), (int)nt, kBT + 2 * R, es, false).end;
        if (smem > (size_t)smem_max) return 0;
        rc = launch_bhm_std<T, R, true>(a, off, b, swept, smem, blocks, s);
    } else {
        const size_t head = (size_t)N * a.n_classes * a.n_classes * es + (size_t)off.n * es;
        const size_t smem = bhm_tail((head + 15) & ~size_t(15), (int)nt, kBT + 2 * R, es, true).end;
        if (smem > (size_t)std::min(smem_max, 160 * 1024)) return 0;
        rc = launch_bhm_std<T, R, false>(a, off, b, swept, smem, blocks, s);
    }
    return rc ? rc : 1;
}

template <typename T>
static int try_bhm_std(const FieldArgs& a, const Offsets& off, int R, const void* wrow, int swept, int smem_max,
                       int blocks, cudaStream_t s) {
    switch (R) {
        case 2: return try_bhm_std_R<T, 2>(a, off, wrow, swept, smem_max, blocks, s);
        case 3: return try_bhm_std_R<T, 3>(a, off, wrow, swept, smem_max, blocks, s);
        case 4: return try_bhm_std_R<T, 4>(a, off, wrow, swept, smem_max, blocks, s);
        case 5: return try_bhm_std_R<T, 5>(a, off, wrow, swept, smem_max, blocks, s);
        default: return 0;
    }
}

template <int R>
static size_t fast_smem(int nk, int nx, int nz, size_t es, bool pn) {
    const int line_max = std::max(nx, nz);
    const size_t LS = ((line_max + 2 * R) + 3) & ~3;
    const size_t tiles = (size_t)((nx + fast::kTile - 1) / fast::kTile) * ((nz + fast::kTile - 1) / fast::kTile);
    return (pn ? 0 : (size_t)nk * nk * fast::Stencil<R>::N * es) + 16 * LS * (2 * es) + 4 * tiles +
           4 * fast::Stencil<R>::N + 4 * (2 * (size_t)nz + 2 * R) + 64;
}

// Row classes of a 2D class map: rowk[z] = the class of every node of row z,
// or -1 if the row holds more than one class.  One CTA per row.
__global__ void row_classes_kernel(const int32_t* __restrict__ cls, int nx, int nz, int* __restrict__ rowk) {
    const int z = blockIdx.x;
    const int32_t* row = cls + (size_t)z * nx;
    const int k0 = row[0];
    bool same = true;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) same = same && row[x] == k0;
    same = __syncthreads_and(same);
    if (threadIdx.x == 0) rowk[z] = same ? k0 : -1;
}

template <typename T, int R, int PPT, bool PN>
static int launch_fast_ppt(const fast::Args& a, size_t smem, int blocks, int threads, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(fast::relax_fast_kernel<T, R, PPT, PN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "relaxation: smem attribute");
    fast::relax_fast_kernel<T, R, PPT, PN><<<blocks, threads, smem, s>>>(a);
    return launch_check("relaxation");
}

// ---- per-node weights -----------------------------------------------------
// Edge-table values [2][n_modes][nk][n_off] (V block, then A block) transposed
// to [2][n_modes][n_off][nk], so that the weight build below reads them along
// the lattice rows when neighbouring nodes have neighbouring classes.
template <typename T>
__global__ void transpose_sel_kernel(const T* __restrict__ in, int nk, int n_off, T* __restrict__ out) {
    __shared__ T tile[32][33];
    const size_t mb = blockIdx.z;                    // block index in [2][n_modes]
    const int k0 = blockIdx.x * 32, o0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, o = o0 + threadIdx.x;
        if (k < nk && o < n_off) tile[r][threadIdx.x] = in[(mb * nk + k) * n_off + o];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int o = o0 + r, k = k0 + threadIdx.x;
        if (k < nk && o < n_off) out[(mb * n_off + o) * nk + k] = tile[threadIdx.x][r];
    }
}

struct StencilArg {
    short x[128], z[128], map[128];
};

// Directed weight of the edge j - o_q -> j for every node j, stencil entry q,
// mode and component (Eq. 28-30, the same rounded operations as the class-pair
// table), written in row layout (z*nx + x) and, through a shared-memory
// transpose, in column layout (x*nz + z).  Edges from outside the lattice get
// +inf.  One 32 x 32 tile of nodes per CTA (32 x 8 threads), all q in turn.
template <typename T>
__global__ void node_weights_kernel(const T* __restrict__ selT, const int32_t* __restrict__ cls, int nx,
                                    int nz, int nk, int n_off, int n_modes, int N, StencilArg st, double dx,
                                    T* __restrict__ wrow, T* __restrict__ wcol) {
    __shared__ T tile[32][33];
    const int mc = blockIdx.z;                       // mode * 2 + component
    const int mode = mc >> 1, comp = mc & 1;
    const T* sel = selT + (size_t)(comp * n_modes + mode) * n_off * nk;
    const int x0 = blockIdx.x * 32, z0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const size_t n = (size_t)nx * nz;
    int kj[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int x = x0 + tx, z = z0 + ty + 8 * r;
        kj[r] = (x < nx && z < nz) ? clamp_class(cls[(size_t)z * nx + x], nk) : 0;
    }
    for (int q = 0; q < N; ++q) {
        const int ox = st.x[q], oz = st.z[q];
        const T L = T(dx * sqrt(double(ox * ox + oz * oz)));
        const T* so = sel + (size_t)st.map[q] * nk;
        T* outr = wrow + ((size_t)mc * N + q) * n;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int x = x0 + tx, z = z0 + ty + 8 * r;
            T w = T(INFINITY);
            if (x < nx && z < nz) {
                const int xi = x - ox, zi = z - oz;
                if (xi >= 0 && xi < nx && zi >= 0 && zi < nz) {
                    const int ki = clamp_class(cls[(size_t)zi * nx + xi], nk);
                    w = edge_w<T>(comp, L, so[ki], so[kj[r]]);
                }
                outr[(size_t)z * nx + x] = w;
            }
            tile[ty + 8 * r][tx] = w;
        }
        __syncthreads();
        T* outc = wcol + ((size_t)mc * N + q) * n;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int x = x0 + ty + 8 * r, z = z0 + tx;
            if (x < nx && z < nz) outc[(size_t)x * nz + z] = tile[tx][ty + 8 * r];
        }
        __syncthreads();
    }
}

// Points per thread of the specialised 2D kernel: 0 = chosen from the line
// length; 1, 2 or 4 = forced where the line fits in 512 threads (set by
// chert_set_relax_points_per_thread, e.g. by an autotuner).
std::atomic<int> g_relax_ppt{0};
std::atomic<int> g_relax3d_tile{0};           // 0: 32 x 16, 1: 64 x 8

// Shared memory of the 3D kernels and their weight mode (1: class-pair table,
// 0: per-class table, 2: tables in global memory) for n_classes classes.
struct Smem3 {
    int mode;
    size_t bytes;
};
static Smem3 smem3(int n_classes, int n_off, int H, int precision, int tile, int smem_max) {
    const size_t es = precision == CHERT_FP64 ? 8 : 4;
    const size_t tas = precision == CHERT_FP32 || precision == CHERT_MIXED ? 4 : 8;   // accumulation type
    const size_t st = tile == 1 ? stage3_elems(H, 64, 8) : stage3_elems(H, 32, 16);
    const size_t base3 = n_off * es + st * (tas + 4) + 4 * 6 * n_off * 2 + 64;
    const size_t t3 = (size_t)n_off * n_classes * n_classes * es + base3;
    const size_t r3 = (size_t)n_classes * n_off * es + base3;
    const int mode = t3 <= (size_t)std::min(smem_max, 160 * 1024) ? 1 : r3 <= (size_t)smem_max ? 0 : 2;
    return {mode, mode == 1 ? t3 : mode == 0 ? r3 : base3};
}

// Whether the offsets are the reach-2 3D table of the unrolled sweeps, in its order.
static bool is_standard3(const Offsets& off) {
    constexpr Stencil3 t{};
    if (off.n != Stencil3::N) return false;
    for (int i = 0; i < Stencil3::N; ++i)
        if (off.x[i] != t.x[i] || off.y[i] != t.y[i] || off.z[i] != t.z[i]) return false;
    return true;
}

// launch_relax3d for the process-wide tile shape and a weight mode
template <typename T, typename TA>
static int launch_relax3d_any(const FieldArgs& a, const Offsets& off, int H, const Smem3& m, int blocks,
                              cudaStream_t s) {
    const int tile = g_relax3d_tile.load();
    if (tile == 1)
        return m.mode == 1 ? launch_relax3d<T, 1, TA, 64, 8>(a, off, H, m.bytes, blocks, s)
             : m.mode == 0 ? launch_relax3d<T, 0, TA, 64, 8>(a, off, H, m.bytes, blocks, s)
                           : launch_relax3d<T, 2, TA, 64, 8>(a, off, H, m.bytes, blocks, s);
    return m.mode == 1 ? launch_relax3d<T, 1, TA, 32, 16>(a, off, H, m.bytes, blocks, s)
         : m.mode == 0 ? launch_relax3d<T, 0, TA, 32, 16>(a, off, H, m.bytes, blocks, s)
                       : launch_relax3d<T, 2, TA, 32, 16>(a, off, H, m.bytes, blocks, s);
}
// 2D scheduler: 0 = ordered sweeps, 1 = block-heap marching, 2 (default) =
// sweeps, then block-heap marching for the fields not yet converged.
std::atomic<int> g_relax_sched{2};
constexpr int kHybridSweeps = 6;

// Radius of the standard stencil with n_off entries (0 if none).
static int standard_radius(int n_off) {
    if (n_off == fast::Stencil<2>::N) return 2;
    if (n_off == fast::Stencil<3>::N) return 3;
    if (n_off == fast::Stencil<4>::N) return 4;
    if (n_off == fast::Stencil<5>::N) return 5;
    return 0;
}

static int max_smem() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 227 * 1024;
    }
    return v;
}

template <int R>
static size_t fast_smem_r(int nk, int nx, int nz, size_t es, bool pn) { return fast_smem<R>(nk, nx, nz, es, pn); }

static size_t fast_smem_any(int R, int nk, int nx, int nz, size_t es, bool pn) {
    switch (R) {
        case 2: return fast_smem_r<2>(nk, nx, nz, es, pn);
        case 3: return fast_smem_r<3>(nk, nx, nz, es, pn);
        case 4: return fast_smem_r<4>(nk, nx, nz, es, pn);
        case 5: return fast_smem_r<5>(nk, nx, nz, es, pn);
        default: return SIZE_MAX;
    }
}

struct PnLayout {
    size_t selT, wrow, wcol, total;    // offsets from the start of the per-node area
};

// Per-node area of the workspace: used by the specialised kernel when the
// stencil is the standard one but the class-pair table does not fit in shared
// memory (e.g. one class per node).  total = 0 when that path does not apply.
static PnLayout pn_layout(int n_modes, int n_classes, int n_off, int precision, int nx, int nz) {
    PnLayout L{0, 0, 0, 0};
    const int R = standard_radius(n_off);
    if (!R || std::max(nx, nz) > 2048) return L;
    const size_t es = precision == CHERT_FP64 ? 8 : 4;
    const int smax = max_smem();
    if (fast_smem_any(R, n_classes, nx, nz, es, false) <= (size_t)smax) return L;   // pair table fits
    if (fast_smem_any(R, n_classes, nx, nz, es, true) > (size_t)smax) return L;
    const size_t m = static_cast<size_t>(n_modes) * n_classes * n_off;
    const size_t wn = static_cast<size_t>(n_modes) * 2 * n_off * nx * nz * es;
    L.selT = 0;
    L.wrow = align256(2 * m * es);
    L.wcol = L.wrow + align256(wn);
    L.total = L.wcol + align256(wn);
    return L;
}

// A 2D lattice prepared for a batched launch of the specialised kernel: its
// arguments (per-node weights and row classes already enqueued) and launch
// shape.
struct FastPrep {
    fast::Args a;
    int R, ppt, threads, blocks;
    bool pn, dbl;
    size_t smem;
};

// Returns 1 if the specialised kernel was launched (or, with prep, set up for
// a batched launch and described in *prep), 0 if the caller must use the
// generic one, or a negative status.  pn_area (pn_bytes long) is the
// workspace's per-node area, or null.
template <typename T, int R>
static int try_fast_R(fast::Args& a, const Offsets& off, int smem_max, int blocks, const void* Vsel,
                      unsigned char* pn_area, size_t pn_bytes, int n_modes, int* rowk_area, cudaStream_t s,
                      FastPrep* prep = nullptr) {
    if (!standard_map<R>(off, a.map)) return 0;
    const int line_max = std::max(a.nx, a.nz);
    if (line_max > 2048) return 0;
    int ppt = line_max <= 512 ? 1 : (line_max <= 1024 ? 2 : 4);
    const int forced = g_relax_ppt.load();
    if ((forced == 1 || forced == 2 || forced == 4) && (line_max + forced - 1) / forced <= 512) ppt = forced;
    const int threads = ((line_max + ppt - 1) / ppt + 31) / 32 * 32;
    size_t smem = fast_smem<R>(a.n_classes, a.nx, a.nz, sizeof(T), false);
    bool pn = false;
    if (smem > (size_t)smem_max) {
        const PnLayout L = pn_layout(n_modes, a.n_classes, off.n, sizeof(T) == 8 ? CHERT_FP64 : CHERT_FP32,
                                     a.nx, a.nz);
        if (!pn_area || L.total == 0 || pn_bytes < L.total) return 0;
        smem = fast_smem<R>(a.n_classes, a.nx, a.nz, sizeof(T), true);
        if (smem > (size_t)smem_max) return 0;
        pn = true;
        constexpr int N = fast::Stencil<R>::N;
        constexpr fast::Stencil<R> st{};
        StencilArg sa;
        for (int q = 0; q < N; ++q) { sa.x[q] = (short)st.x[q]; sa.z[q] = (short)st.z[q]; sa.map[q] = a.map[q]; }
        T* selT = reinterpret_cast<T*>(pn_area + L.selT);
        transpose_sel_kernel<T><<<dim3((a.n_classes + 31) / 32, (off.n + 31) / 32, 2 * n_modes), dim3(32, 8), 0, s>>>(
            static_cast<const T*>(Vsel), a.n_classes, off.n, selT);
        int rc = launch_check("relaxation: edge-table transpose");
        if (rc) return rc;
        T* wr = reinterpret_cast<T*>(pn_area + L.wrow);
        T* wc = reinterpret_cast<T*>(pn_area + L.wcol);
        node_weights_kernel<T><<<dim3((a.nx + 31) / 32, (a.nz + 31) / 32, 2 * n_modes), dim3(32, 8), 0, s>>>(
            selT, a.cls, a.nx, a.nz, a.n_classes, off.n, n_modes, N, sa, a.dx, wr, wc);
        rc = launch_check("relaxation: per-node weights");
        if (rc) return rc;
        a.wrow = wr;
        a.wcol = wc;
    } else {
        a.wrow = a.wcol = nullptr;
    }
    a.rowk = nullptr;
    if (!pn && rowk_area && a.nz <= kRowkMax) {        // row-class path, if every row is one class
        row_classes_kernel<<<a.nz, 128, 0, s>>>(a.cls, a.nx, a.nz, rowk_area);
        const int rc0 = launch_check("relaxation: row classes");
        if (rc0) return rc0;
        a.rowk = rowk_area;
    }
    if (prep) {
        prep->a = a;
        prep->R = R;
        prep->ppt = ppt;
        prep->threads = threads;
        prep->blocks = blocks;
        prep->pn = pn;
        prep->dbl = sizeof(T) == 8;
        prep->smem = smem;
        return 1;
    }
    int rc;
    if (pn)
        rc = ppt == 1 ? launch_fast_ppt<T, R, 1, true>(a, smem, blocks, threads, s)
           : ppt == 2 ? launch_fast_ppt<T, R, 2, true>(a, smem, blocks, threads, s)
                      : launch_fast_ppt<T, R, 4, true>(a, smem, blocks, threads, s);
    else
        rc = ppt == 1 ? launch_fast_ppt<T, R, 1, false>(a, smem, blocks, threads, s)
           : ppt == 2 ? launch_fast_ppt<T, R, 2, false>(a, smem, blocks, threads, s)
                      : launch_fast_ppt<T, R, 4, false>(a, smem, blocks, threads, s);
    return rc ? rc : 1;
}

template <typename T>
static int try_fast(fast::Args& a, const Offsets& off, int R, int smem_max, int blocks, const void* Vsel,
                    unsigned char* pn_area, size_t pn_bytes, int n_modes, int* rowk_area, cudaStream_t s,
                    FastPrep* prep = nullptr) {
    switch (R) {
        case 2: return try_fast_R<T, 2>(a, off, smem_max, blocks, Vsel, pn_area, pn_bytes, n_modes, rowk_area, s, prep);
        case 3: return try_fast_R<T, 3>(a, off, smem_max, blocks, Vsel, pn_area, pn_bytes, n_modes, rowk_area, s, prep);
        case 4: return try_fast_R<T, 4>(a, off, smem_max, blocks, Vsel, pn_area, pn_bytes, n_modes, rowk_area, s, prep);
        case 5: return try_fast_R<T, 5>(a, off, smem_max, blocks, Vsel, pn_area, pn_bytes, n_modes, rowk_area, s, prep);
        default: return 0;
    }
}

extern "C" size_t chert_traveltime_workspace_bytes(int n_modes, int n_classes, int n_off,
                                                   int precision, int n_sources) {
    if (n_modes < 1 || n_classes < 1 || n_off < 1 || n_sources < 1) return 0;
    return ws_layout(n_modes, n_classes, n_off, precision, n_sources).total;
}

extern "C" size_t chert_traveltime_workspace_bytes_grid(int n_modes, int n_classes, int n_off, int precision,
                                                        int n_sources, int nx, int ny, int nz) {
    if (n_modes < 1 || n_classes < 1 || n_off < 1 || n_sources < 1 || nx < 1 || ny < 1 || nz < 1) return 0;
    if (ny > 1) return ws_layout(n_modes, n_classes, n_off, precision, n_sources).total;   // 3D: no per-node area
    return ws_layout(n_modes, n_classes, n_off, precision, n_sources).total +
           pn_layout(n_modes, n_classes, n_off, precision, nx, nz).total;
}

// Validates the arguments and enqueues lookup, class check and relaxation on
// `s`, using `w` (bytes long) as scratch.  On success *blocks_out is the number
// of relaxation CTAs and *status_out points at their status words (followed by
// the class-check flag), which the caller reads back.
// A lattice prepared (edge tables, class check, status) for a batched launch:
// 3D (FieldArgs, halo H) or 2D (fast2d set, fast2d_ok = 1 when the
// specialised kernel takes it; 0: the caller relaxes it on its own).
struct Prep3 {
    FieldArgs a;
    int H, blocks;
    FastPrep fast2d;
    int fast2d_ok;
};

static int enqueue_traveltime(const char* who, const chert_cache_arrays* cache, int n_modes,
                              int n_classes, int n_dir, int nx, int ny, int nz, double dx,
                              const int32_t* d_class_of_node, const int32_t* offsets, int n_off,
                              const int64_t* sources, int n_sources, int precision, int max_cycles,
                              void* d_tauR, void* d_tauI, int32_t* d_parR, int32_t* d_parI,
                              unsigned char* w, size_t bytes, cudaStream_t s, int* blocks_out,
                              int** status_out, const int64_t* d_sources = nullptr, Prep3* prep = nullptr) {
    CHERT_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1 && (long long)nx * ny * nz < (1LL << 31),
                  "%s: bad lattice %d x %d x %d", who, nx, ny, nz);
    const long long n_nodes = (long long)nx * ny * nz;
    CHERT_REQUIRE(dx > 0, "%s: dx must be positive", who);
    CHERT_REQUIRE(d_class_of_node && (sources || d_sources) && d_tauR && d_tauI && w, "%s: NULL argument", who);
    CHERT_REQUIRE(n_sources >= 1 && n_modes >= 1 && n_modes <= 3 && n_classes >= 1,
                  "%s: bad counts", who);
    CHERT_REQUIRE(max_cycles >= 1, "%s: max_cycles must be >= 1", who);
    CHERT_REQUIRE(precision == CHERT_FP64 || precision == CHERT_FP32 || precision == CHERT_MIXED ||
                      precision == CHERT_FP32_ACC64,
                  "%s: precision=%d", who, precision);
    CHERT_REQUIRE(precision != CHERT_FP32_ACC64 || ny > 1,
                  "%s: CHERT_FP32_ACC64 is for 3D lattices (ny > 1)", who);
    for (int i = 0; sources && i < n_sources; i++)
        CHERT_REQUIRE(sources[i] >= 0 && sources[i] < (int64_t)n_nodes,
                      "%s: source %d out of range", who, i);
    Offsets off;
    int rc = fill_offsets(off, offsets, n_off, who);
    if (rc) return rc;
    int R = 0;
    for (int i = 0; i < n_off; i++) {
        CHERT_REQUIRE(ny > 1 || off.y[i] == 0, "%s: 2D offsets need oy = 0", who);
        R = std::max(R, std::max(abs((int)off.x[i]), abs((int)off.z[i])));
        bool has_neg = false;
        for (int j = 0; j < n_off; j++)
            if (off.x[j] == -off.x[i] && off.y[j] == -off.y[i] && off.z[j] == -off.z[i]) has_neg = true;
        CHERT_REQUIRE(has_neg, "%s: offset set must be closed under negation", who);
    }
    const WsLayout ws = ws_layout(n_modes, n_classes, n_off, precision, n_sources);
    if (bytes < ws.total) {
        set_error("%s: workspace %zu < %zu bytes", who, bytes, ws.total);
        return CHERT_ENOMEM;
    }
    const size_t es = precision == CHERT_FP64 ? 8 : 4;
    const size_t m = static_cast<size_t>(n_modes) * n_classes * n_off;
    void* Vsel = w + ws.sel;
    void* Asel = w + ws.sel + m * es;
    rc = chert_edge_table(cache, n_modes, n_classes, n_dir, precision == CHERT_FP32_ACC64 ? CHERT_FP32 : precision,
                          offsets, n_off,
                          reinterpret_cast<int32_t*>(w + ws.idx), Vsel, Asel, s);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (sources) {
        e = cudaMemcpyAsync(w + ws.src, sources, sizeof(int64_t) * n_sources, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "sources copy");
    }

    int* bad_class = reinterpret_cast<int*>(w + ws.status) + (size_t)n_sources * n_modes * 2;
    e = cudaMemsetAsync(bad_class, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    check_classes_kernel<<<296, 256, 0, s>>>(d_class_of_node, n_nodes, n_classes, bad_class);
    rc = launch_check("class check");
    if (rc) return rc;

    FieldArgs a;
    a.nx = nx; a.ny = ny; a.nz = nz; a.n_classes = n_classes; a.n_modes = n_modes;
    a.n_sources = n_sources; a.max_cycles = max_cycles; a.ring = R + 2; a.dx = dx;
    a.cls = d_class_of_node;
    a.src = d_sources ? d_sources : reinterpret_cast<const int64_t*>(w + ws.src);
    a.tauR = d_tauR; a.tauI = d_tauI; a.parR = d_parR; a.parI = d_parI;
    a.Vsel = Vsel; a.Asel = Asel; a.status = reinterpret_cast<int*>(w + ws.status);
    a.parts = 1;
    a.sync = reinterpret_cast<unsigned*>(w + ws.sync);
    a.std3 = 0;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int blocks = n_sources * n_modes * 2;
    if (ny > 1) {                                      // 3D: plane sweeps
        int H = 0;
        for (int i = 0; i < n_off; i++)
            H = std::max(H, std::max(abs((int)off.y[i]), std::max(abs((int)off.x[i]), abs((int)off.z[i]))));
        CHERT_REQUIRE(H <= 8, "%s: 3D offsets reach %d nodes (at most 8)", who, H);
        a.std3 = H == 2 && is_standard3(off) ? 1 : 0;
        const Smem3 m3 = smem3(n_classes, n_off, H, precision, g_relax3d_tile.load(), smem_max);
        if (prep) {                                    // a batched launch runs the relaxation
            prep->a = a;
            prep->H = H;
            prep->blocks = blocks;
            return CHERT_OK;
        }
        if (precision == CHERT_FP32_ACC64)
            rc = launch_relax3d_any<float, xf::ff>(a, off, H, m3, blocks, s);
        else if (precision == CHERT_FP64)
            rc = launch_relax3d_any<double, double>(a, off, H, m3, blocks, s);
        else
            rc = launch_relax3d_any<float, float>(a, off, H, m3, blocks, s);
        if (rc) return rc;
        *blocks_out = blocks;
        *status_out = a.status;
        return CHERT_OK;
    }
    if (prep) {
        // a batched launch (chert_traveltime_batch): the sweeps of the
        // specialised kernel, set up here and launched with the batch
        fast::Args fa;
        fa.nx = nx; fa.nz = nz; fa.n_classes = n_classes; fa.n_modes = n_modes;
        fa.max_cycles = max_cycles; fa.dx = dx; fa.cls = a.cls; fa.src = a.src;
        fa.tauR = d_tauR; fa.tauI = d_tauI; fa.parR = d_parR; fa.parI = d_parI;
        fa.Vsel = Vsel; fa.Asel = Asel; fa.n_off = n_off; fa.status = a.status;
        fa.wrow = fa.wcol = nullptr;
        unsigned char* pn_area = bytes > ws.total ? w + ws.total : nullptr;
        const size_t pn_bytes = bytes > ws.total ? bytes - ws.total : 0;
        int* rowk_area = reinterpret_cast<int*>(w + ws.rowk);
        const int fr = precision == CHERT_FP64
                           ? try_fast<double>(fa, off, R, smem_max, blocks, Vsel, pn_area, pn_bytes, n_modes,
                                              rowk_area, s, &prep->fast2d)
                           : try_fast<float>(fa, off, R, smem_max, blocks, Vsel, pn_area, pn_bytes, n_modes,
                                             rowk_area, s, &prep->fast2d);
        if (fr < 0) return fr;
        prep->fast2d_ok = fr;
        prep->a = a;
        prep->H = 0;
        prep->blocks = blocks;
        return CHERT_OK;
    }
    // 2D schedulers: 0 sweeps; 1 block-heap marching; 2 sweeps for at most
    // kHybridSweeps cycles, then block-heap marching, from the source, for
    // the fields that did not converge.
    const int sched = g_relax_sched.load();
    CHERT_REQUIRE(sched != 1 || R <= kBH, "%s: the block scheduler takes stencils of reach <= %d (got %d)", who,
                  kBH, R);
    if (sched == 3) {                                  // frontier label correcting
        const size_t wb = ((size_t)n_off * n_classes * n_classes * es + 15) & ~size_t(15);
        const size_t smf = wb + 2 * 4 * (((size_t)nx * nz + 31) / 32);
        CHERT_REQUIRE(smf <= (size_t)smem_max,
                      "%s: the frontier scheduler needs the class-pair table and two bitmaps in shared memory "
                      "(%zu > %d bytes)", who, smf, smem_max);
        frontier::Args fa;
        fa.nx = nx; fa.nz = nz; fa.n_classes = n_classes; fa.n_modes = n_modes;
        fa.max_rounds = max_cycles * std::max(nx, nz);
        fa.dx = dx; fa.cls = a.cls; fa.src = a.src;
        fa.tauR = d_tauR; fa.tauI = d_tauI; fa.parR = d_parR; fa.parI = d_parI;
        fa.Vsel = Vsel; fa.Asel = Asel; fa.status = a.status;
        const bool dbl = precision == CHERT_FP64;
        cudaError_t e2 = dbl ? cudaFuncSetAttribute(relax_frontier_kernel<double>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf)
                             : cudaFuncSetAttribute(relax_frontier_kernel<float>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
        if (e2 != cudaSuccess) return cuda_fail(e2, "chert_traveltime: smem attribute");
        if (dbl)
            relax_frontier_kernel<double><<<blocks, 1024, smf, s>>>(fa, off);
        else
            relax_frontier_kernel<float><<<blocks, 1024, smf, s>>>(fa, off);
        rc = launch_check("chert_traveltime: frontier");
        if (rc) return rc;
        *blocks_out = blocks;
        *status_out = a.status;
        return CHERT_OK;
    }
    const bool hybrid = sched == 2 && R <= kBH && max_cycles > kHybridSweeps;
    const void* swept_wrow = nullptr;                  // per-node weights the sweeps computed, if any
    auto block_heap = [&](int swept) -> int {
        const int r = precision == CHERT_FP64
                          ? try_bhm_std<double>(a, off, R, swept_wrow, swept, smem_max, blocks, s)
                          : try_bhm_std<float>(a, off, R, swept_wrow, swept, smem_max, blocks, s);
        if (r < 0) return r;
        if (r == 1) return CHERT_OK;
        const size_t nt = (size_t)((nx + kBT - 1) / kBT) * ((nz + kBT - 1) / kBT);
        auto tail = [&](size_t wbytes) {
            const size_t head = wbytes + n_off * es + (size_t)n_off * 4;
            return bhm_tail((head + 15) & ~size_t(15), (int)nt, kBT + 2 * R, es, true).end;
        };
        const size_t baseb = tail(0);
        const size_t tb = tail((size_t)n_off * n_classes * n_classes * es);
        const size_t rb = tail((size_t)n_classes * n_off * es);
        const int mb = tb <= (size_t)std::min(smem_max, 160 * 1024) ? 1 : rb <= (size_t)smem_max ? 0 : 2;
        const size_t smb = mb == 1 ? tb : mb == 0 ? rb : baseb;
        CHERT_REQUIRE(smb <= (size_t)smem_max, "%s: lattice too large for the block scheduler", who);
        if (precision == CHERT_FP64)
            return mb == 1 ? launch_bhm<double, 1>(a, off, R, swept, smb, blocks, s)
                 : mb == 0 ? launch_bhm<double, 0>(a, off, R, swept, smb, blocks, s)
                           : launch_bhm<double, 2>(a, off, R, swept, smb, blocks, s);
        return mb == 1 ? launch_bhm<float, 1>(a, off, R, swept, smb, blocks, s)
             : mb == 0 ? launch_bhm<float, 0>(a, off, R, swept, smb, blocks, s)
                       : launch_bhm<float, 2>(a, off, R, swept, smb, blocks, s);
    };
    if (sched == 1) {
        rc = block_heap(0);
        if (rc) return rc;
        *blocks_out = blocks;
        *status_out = a.status;
        return CHERT_OK;
    }
    const int sweep_cycles = hybrid ? kHybridSweeps : max_cycles;
    a.max_cycles = sweep_cycles;
    const int line_max = std::max(nx, nz);
    const size_t common = n_off * es + (size_t)a.ring * line_max * (es + 4) + 4 * n_off * 2 + 32;
    const size_t smem_table = (size_t)n_off * n_classes * n_classes * es + common;
    const size_t smem_raw = (size_t)n_classes * n_off * es + common;
    const bool table = smem_table <= (size_t)std::min(smem_max, 120 * 1024);
    const bool raw_smem = smem_raw <= (size_t)smem_max;
    fast::Args fa;
    fa.nx = nx; fa.nz = nz; fa.n_classes = n_classes; fa.n_modes = n_modes;
    fa.max_cycles = sweep_cycles; fa.dx = dx; fa.cls = a.cls; fa.src = a.src;
    fa.tauR = d_tauR; fa.tauI = d_tauI; fa.parR = d_parR; fa.parI = d_parI;
    fa.Vsel = Vsel; fa.Asel = Asel; fa.n_off = n_off; fa.status = a.status;
    fa.wrow = fa.wcol = nullptr;
    unsigned char* pn_area = bytes > ws.total ? w + ws.total : nullptr;
    const size_t pn_bytes = bytes > ws.total ? bytes - ws.total : 0;
    int* rowk_area = reinterpret_cast<int*>(w + ws.rowk);
    const int fr = precision == CHERT_FP64
                       ? try_fast<double>(fa, off, R, smem_max, blocks, Vsel, pn_area, pn_bytes, n_modes, rowk_area, s)
                       : try_fast<float>(fa, off, R, smem_max, blocks, Vsel, pn_area, pn_bytes, n_modes, rowk_area, s);
    if (fr < 0) return fr;
    if (fr == 1) rc = CHERT_OK;
    else if (precision == CHERT_FP64)
        rc = table ? launch_relax<double, 1>(a, off, smem_table, blocks, s)
           : raw_smem ? launch_relax<double, 0>(a, off, smem_raw, blocks, s)
                      : launch_relax<double, 2>(a, off, common, blocks, s);
    else
        rc = table ? launch_relax<float, 1>(a, off, smem_table, blocks, s)
           : raw_smem ? launch_relax<float, 0>(a, off, smem_raw, blocks, s)
                      : launch_relax<float, 2>(a, off, common, blocks, s);
    if (rc) return rc;
    if (hybrid) {
        a.max_cycles = max_cycles;
        swept_wrow = fa.wrow;
        rc = block_heap(kHybridSweeps);
        if (rc) return rc;
    }
    *blocks_out = blocks;
    *status_out = a.status;
    return CHERT_OK;
}

static int status_to_code(const char* who, int first_bad_block, int bad_class, int n_classes,
                          int max_cycles) {
    if (bad_class) {
        set_error("%s: class map holds ids outside [0, %d)", who, n_classes);
        return CHERT_EINVAL;
    }
    if (first_bad_block >= 0) {
        set_error("%s: field %d component %d did not converge in %d cycles", who,
                  first_bad_block / 2, first_bad_block % 2, max_cycles);
        return CHERT_ETIMEOUT;
    }
    return CHERT_OK;
}

extern "C" int chert_traveltime(const chert_cache_arrays* cache, int n_modes, int n_classes,
                                int n_dir, int nx, int ny, int nz, double dx,
                                const int32_t* d_class_of_node, const int32_t* offsets, int n_off,
                                const int64_t* sources, int n_sources, int precision,
                                int max_cycles, void* d_tauR, void* d_tauI, int32_t* d_parR,
                                int32_t* d_parI, void* d_workspace, size_t workspace_bytes,
                                void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int blocks = 0;
    int* status = nullptr;
    int rc = enqueue_traveltime("chert_traveltime", cache, n_modes, n_classes, n_dir, nx, ny, nz,
                                dx, d_class_of_node, offsets, n_off, sources, n_sources, precision,
                                max_cycles, d_tauR, d_tauI, d_parR, d_parI,
                                static_cast<unsigned char*>(d_workspace), workspace_bytes, s,
                                &blocks, &status);
    if (rc) return rc;
    // convergence status: one int per CTA, then the class-check flag
    int* host_status = static_cast<int*>(malloc(sizeof(int) * (blocks + 1)));
    if (!host_status) { set_error("chert_traveltime: host malloc"); return CHERT_ENOMEM; }
    cudaError_t e = cudaMemcpyAsync(host_status, status, sizeof(int) * (blocks + 1),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { free(host_status); return cuda_fail(e, "chert_traveltime: status"); }
    int bad = -1;
    for (int b = 0; b < blocks; b++) if (host_status[b] < 0) { bad = b; break; }
    const int bad_cls = host_status[blocks];
    free(host_status);
    return status_to_code("chert_traveltime", bad, bad_cls, n_classes, max_cycles);
}

// ------------------------------------------------------------------------
// chert_traveltime_static: the same relaxation for callers that must not
// allocate device memory (an allocator-free embedding, a host that has handed
// all device memory to its own pool).  Its scratch is the file-scope array
// below instead of a caller-provided workspace; every device that loads
// libchert keeps the array for the life of the process.
namespace chert {
namespace {
constexpr size_t kStaticScratchBytes = size_t(1) << 20;     // 1 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once
// per device (the host-side symbol is not a device address) and kept for the
// life of the process: a cudaDeviceReset of the device makes it stale.
int static_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime_static: cudaGetDevice");
    CHERT_REQUIRE(dev >= 0 && dev < kMaxDevices, "chert_traveltime_static: device %d", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (g_static_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime_static: cudaGetSymbolAddress");
        g_static_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_static_ptr[dev]);
    return CHERT_OK;
}

// One block: summary[0] = first CTA that hit the cycle cap (or -1),
// summary[1] = class-check flag.  Written on every call.
__global__ void status_summary_kernel(const int* __restrict__ status, int n_blocks,
                                      int* __restrict__ summary) {
    __shared__ int first;
    if (threadIdx.x == 0) first = INT_MAX;
    __syncthreads();
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x)
        if (status[b] < 0) atomicMin(&first, b);
    __syncthreads();
    if (threadIdx.x == 0) {
        summary[0] = first == INT_MAX ? -1 : first;
        summary[1] = status[n_blocks];
    }
}
}  // namespace
}  // namespace chert

extern "C" size_t chert_traveltime_static_limit(void) { return chert::kStaticScratchBytes; }

extern "C" int chert_traveltime_static(const chert_cache_arrays* cache, int n_modes, int n_classes,
                                       int n_dir, int nx, int ny, int nz, double dx,
                                       const int32_t* d_class_of_node, const int32_t* offsets,
                                       int n_off, const int64_t* sources, int n_sources,
                                       int precision, int max_cycles, void* d_tauR, void* d_tauI,
                                       int32_t* d_parR, int32_t* d_parI, void* stream) {
    CHERT_REQUIRE(n_modes >= 1 && n_classes >= 1 && n_off >= 1 && n_sources >= 1,
                  "chert_traveltime_static: bad counts");
    const size_t need = ws_layout(n_modes, n_classes, n_off, precision, n_sources).total;
    const size_t summary_at = kStaticScratchBytes - 256;
    CHERT_REQUIRE(need <= summary_at,
                  "chert_traveltime_static: this problem needs %zu bytes of scratch; the static "
                  "scratch holds %zu (use chert_traveltime with a workspace)",
                  need, summary_at);
    unsigned char* w = nullptr;
    int rc = static_scratch(&w);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int blocks = 0;
    int* status = nullptr;
    rc = enqueue_traveltime("chert_traveltime_static", cache, n_modes, n_classes, n_dir, nx, ny, nz,
                            dx, d_class_of_node, offsets, n_off, sources, n_sources, precision,
                            max_cycles, d_tauR, d_tauI, d_parR, d_parI, w, summary_at, s, &blocks,
                            &status);
    if (rc) return rc;
    int* summary = reinterpret_cast<int*>(w + summary_at);
    status_summary_kernel<<<1, 256, 0, s>>>(status, blocks, summary);
    rc = launch_check("chert_traveltime_static: status");
    if (rc) return rc;
    int h[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, summary, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime_static: status");
    return status_to_code("chert_traveltime_static", h[0], h[1], n_classes, max_cycles);
}

// chert_traveltime_enqueue: the same path with device sources and a device
// status word pair, and no host synchronisation or host-to-device copy.
extern "C" int chert_traveltime_enqueue(const chert_cache_arrays* cache, int n_modes, int n_classes, int n_dir,
                                        int nx, int ny, int nz, double dx, const int32_t* d_class_of_node,
                                        const int32_t* offsets, int n_off, const int64_t* d_sources,
                                        int n_sources, int precision, int max_cycles, void* d_tauR,
                                        void* d_tauI, int32_t* d_parR, int32_t* d_parI, void* d_workspace,
                                        size_t workspace_bytes, int32_t* d_status, void* stream) {
    CHERT_REQUIRE(d_sources && d_status, "chert_traveltime_enqueue: NULL sources or status");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int blocks = 0;
    int* status = nullptr;
    int rc = enqueue_traveltime("chert_traveltime_enqueue", cache, n_modes, n_classes, n_dir, nx, ny, nz, dx,
                                d_class_of_node, offsets, n_off, nullptr, n_sources, precision, max_cycles,
                                d_tauR, d_tauI, d_parR, d_parI, static_cast<unsigned char*>(d_workspace),
                                workspace_bytes, s, &blocks, &status, d_sources);
    if (rc) return rc;
    status_summary_kernel<<<1, 256, 0, s>>>(status, blocks, d_status);
    return launch_check("chert_traveltime_enqueue: status");
}

template <typename T, typename TA, int TU, int TV>
static int launch_multi3d(const LatticeTable& t, const Offsets& off, int H, const Smem3& m, long long items,
                          unsigned long long* counter, cudaStream_t s) {
    auto k = m.mode == 1 ? relax3d_multi_kernel<T, TA, 1, TU, TV>
           : m.mode == 0 ? relax3d_multi_kernel<T, TA, 0, TU, TV>
                         : relax3d_multi_kernel<T, TA, 2, TU, TV>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m.bytes);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime_batch: smem attribute");
    int dev = 0, n_sm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 512, m.bytes) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        n_sm = 148;
        per_sm = 1;
    }
    const long long grid = std::min<long long>(items, (long long)n_sm * per_sm);   // persistent: one wave
    k<<<(unsigned)grid, 512, m.bytes, s>>>(t, off, H, counter);
    return launch_check("chert_traveltime_batch: relax3d (persistent)");
}

// One persistent launch of 2D lattices that share a launch shape (radius-5
// stencil, nodes a thread, weight form, precision): at most
// kMaxFastLattices of them.
template <typename T, int PPT, bool PN>
static int launch_multi2d(const fast::FastTable& t, int threads, size_t smem, long long items,
                          unsigned long long* counter, cudaStream_t s) {
    auto k = fast::relax_fast_multi_kernel<T, 5, PPT, PN>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime_batch: smem attribute");
    int dev = 0, n_sm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        n_sm = 148;
        per_sm = 1;
    }
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime_batch: counter");
    const long long grid = std::min<long long>(items, (long long)n_sm * per_sm);   // persistent: one wave
    k<<<(unsigned)grid, threads, smem, s>>>(t, counter);
    return launch_check("chert_traveltime_batch: relax_fast (persistent)");
}

// The 2D lattices of a batch: the ones the specialised kernel takes with the
// radius-5 stencil are grouped by launch shape, each group one persistent
// launch (of at most kMaxFastLattices lattices); the others are relaxed on
// their own, as chert_traveltime_enqueue relaxes them.
static int batch_2d(const chert_lattice* lattices, int n_lattices, int n_modes, int precision,
                    const int32_t* offsets, int n_off, int max_cycles, std::vector<Prep3>& prep,
                    unsigned long long* d_counter, cudaStream_t s) {
    std::vector<int> alone, grouped;
    for (int i = 0; i < n_lattices; ++i)
        (prep[i].fast2d_ok == 1 && prep[i].fast2d.R == 5 ? grouped : alone).push_back(i);
    for (int i : alone) {
        const chert_lattice& L = lattices[i];
        const int rc = chert_traveltime_enqueue(L.cache, n_modes, L.n_classes, L.n_dir, L.nx, 1, L.nz, L.dx,
                                                L.d_class_of_node, offsets, n_off, L.d_sources, L.n_sources,
                                                precision, max_cycles, L.d_tauR, L.d_tauI, L.d_parR, L.d_parI,
                                                L.d_workspace, L.workspace_bytes, L.d_status, s);
        if (rc) return rc;
    }
    // largest lattices first
    std::stable_sort(grouped.begin(), grouped.end(), [&](int x, int y) {
        const fast::Args &a = prep[x].fast2d.a, &b = prep[y].fast2d.a;
        return (long long)a.nx * a.nz > (long long)b.nx * b.nz;
    });
    std::vector<char> done(n_lattices, 0);
    for (size_t g0 = 0; g0 < grouped.size(); ++g0) {
        const int lead = grouped[g0];
        if (done[lead]) continue;
        const FastPrep& P = prep[lead].fast2d;
        std::vector<int> members;
        for (size_t g = g0; g < grouped.size() && (int)members.size() < fast::kMaxFastLattices; ++g) {
            const FastPrep& Q = prep[grouped[g]].fast2d;
            if (!done[grouped[g]] && Q.ppt == P.ppt && Q.pn == P.pn && Q.dbl == P.dbl) {
                members.push_back(grouped[g]);
                done[grouped[g]] = 1;
            }
        }
        fast::FastTable t;
        t.n = (int)members.size();
        long long at = 0;
        int threads = 32;
        size_t smem = 0;
        for (int m = 0; m < t.n; ++m) {            // attenuation components of every lattice
            const FastPrep& Q = prep[members[m]].fast2d;
            t.a[m] = Q.a;
            t.start[m] = at;
            at += Q.blocks / 2;
            threads = std::max(threads, Q.threads);
            smem = std::max(smem, Q.smem);
        }
        for (int m = 0; m < t.n; ++m) {            // then the propagation components
            t.start[t.n + m] = at;
            at += prep[members[m]].fast2d.blocks / 2;
        }
        t.start[2 * t.n] = at;
        int rc;
        if (P.dbl)
            rc = P.pn ? (P.ppt == 1 ? launch_multi2d<double, 1, true>(t, threads, smem, at, d_counter, s)
                       : P.ppt == 2 ? launch_multi2d<double, 2, true>(t, threads, smem, at, d_counter, s)
                                    : launch_multi2d<double, 4, true>(t, threads, smem, at, d_counter, s))
                      : (P.ppt == 1 ? launch_multi2d<double, 1, false>(t, threads, smem, at, d_counter, s)
                       : P.ppt == 2 ? launch_multi2d<double, 2, false>(t, threads, smem, at, d_counter, s)
                                    : launch_multi2d<double, 4, false>(t, threads, smem, at, d_counter, s));
        else
            rc = P.pn ? (P.ppt == 1 ? launch_multi2d<float, 1, true>(t, threads, smem, at, d_counter, s)
                       : P.ppt == 2 ? launch_multi2d<float, 2, true>(t, threads, smem, at, d_counter, s)
                                    : launch_multi2d<float, 4, true>(t, threads, smem, at, d_counter, s))
                      : (P.ppt == 1 ? launch_multi2d<float, 1, false>(t, threads, smem, at, d_counter, s)
                       : P.ppt == 2 ? launch_multi2d<float, 2, false>(t, threads, smem, at, d_counter, s)
                                    : launch_multi2d<float, 4, false>(t, threads, smem, at, d_counter, s));
        if (rc) return rc;
    }
    for (int i : grouped)
        status_summary_kernel<<<1, 256, 0, s>>>(prep[i].a.status, prep[i].blocks, lattices[i].d_status);
    return launch_check("chert_traveltime_batch: status");
}

extern "C" int chert_traveltime_batch(const chert_lattice* lattices, int n_lattices, int n_modes, int precision,
                                      const int32_t* offsets, int n_off, int max_cycles,
                                      unsigned long long* d_counter, void* stream) {
    const char* who = "chert_traveltime_batch";
    CHERT_REQUIRE(lattices && offsets && d_counter, "%s: NULL argument", who);
    CHERT_REQUIRE(n_lattices >= 1 && n_lattices <= kMaxLattices, "%s: n_lattices=%d (1..%d)", who, n_lattices,
                  kMaxLattices);
    CHERT_REQUIRE(precision == CHERT_FP64 || precision == CHERT_FP32 || precision == CHERT_MIXED ||
                      precision == CHERT_FP32_ACC64, "%s: precision=%d", who, precision);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<Prep3> prep(n_lattices);
    int max_nk = 1;
    const bool two_d = lattices[0].ny == 1;
    for (int i = 0; i < n_lattices; ++i) {
        const chert_lattice& L = lattices[i];
        CHERT_REQUIRE(L.cache && L.d_sources && L.d_status, "%s: lattice %d: NULL cache, sources or status", who, i);
        CHERT_REQUIRE((L.ny == 1) == two_d, "%s: lattice %d: a batch is all 2D (ny = 1) or all 3D", who, i);
        CHERT_REQUIRE(L.ny >= 1, "%s: lattice %d: ny=%d", who, i, L.ny);
        prep[i].fast2d_ok = 0;
        int blocks = 0;
        int* st = nullptr;
        const int rc = enqueue_traveltime(who, L.cache, n_modes, L.n_classes, L.n_dir, L.nx, L.ny, L.nz, L.dx,
                                          L.d_class_of_node, offsets, n_off, nullptr, L.n_sources, precision,
                                          max_cycles, L.d_tauR, L.d_tauI, L.d_parR, L.d_parI,
                                          static_cast<unsigned char*>(L.d_workspace), L.workspace_bytes, s, &blocks,
                                          &st, L.d_sources, &prep[i]);
        if (rc) return rc;
        prep[i].a.parts = 1;
        max_nk = std::max(max_nk, L.n_classes);
    }
    if (two_d)
        return batch_2d(lattices, n_lattices, n_modes, precision, offsets, n_off, max_cycles, prep, d_counter, s);
    // largest lattices first, so that the longest items start first
    std::vector<int> order(n_lattices);
    for (int i = 0; i < n_lattices; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const FieldArgs &a = prep[x].a, &b = prep[y].a;
        return (long long)a.nx * a.ny * a.nz > (long long)b.nx * b.ny * b.nz;
    });
    LatticeTable t;
    t.n = n_lattices;
    t.start[0] = 0;
    for (int i = 0; i < n_lattices; ++i) {
        t.a[i] = prep[order[i]].a;
        t.start[i + 1] = t.start[i] + prep[order[i]].blocks;
    }
    Offsets off;
    int rc = fill_offsets(off, offsets, n_off, who);
    if (rc) return rc;
    const int H = prep[0].H;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int tile = g_relax3d_tile.load();
    const Smem3 m = smem3(max_nk, n_off, H, precision, tile, smem_max);
    cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "chert_traveltime_batch: counter");
    const long long items = t.start[n_lattices];
    if (precision == CHERT_FP32_ACC64)
        rc = tile == 1 ? launch_multi3d<float, xf::ff, 64, 8>(t, off, H, m, items, d_counter, s)
                       : launch_multi3d<float, xf::ff, 32, 16>(t, off, H, m, items, d_counter, s);
    else if (precision == CHERT_FP64)
        rc = tile == 1 ? launch_multi3d<double, double, 64, 8>(t, off, H, m, items, d_counter, s)
                       : launch_multi3d<double, double, 32, 16>(t, off, H, m, items, d_counter, s);
    else
        rc = tile == 1 ? launch_multi3d<float, float, 64, 8>(t, off, H, m, items, d_counter, s)
                       : launch_multi3d<float, float, 32, 16>(t, off, H, m, items, d_counter, s);
    if (rc) return rc;
    for (int i = 0; i < n_lattices; ++i)
        status_summary_kernel<<<1, 256, 0, s>>>(prep[i].a.status, prep[i].blocks, lattices[i].d_status);
    return launch_check("chert_traveltime_batch: status");
}

extern "C" int chert_set_relax3d_tile(int tile) {
    CHERT_REQUIRE(tile == 0 || tile == 1, "chert_set_relax3d_tile: tile=%d (0: 32 x 16, 1: 64 x 8)", tile);
    return g_relax3d_tile.exchange(tile);
}

extern "C" int chert_raypath(const int32_t* d_par, int n_fields, int64_t n_nodes,
                             const int64_t* d_src, const int64_t* d_rcv, int n_rcv, int64_t cap,
                             int64_t* d_paths, int64_t* d_len, void* stream) {
    CHERT_REQUIRE(d_par && d_src && d_rcv && d_paths && d_len, "chert_raypath: NULL argument");
    CHERT_REQUIRE(n_fields >= 1 && n_nodes >= 1 && n_rcv >= 1 && cap >= 1,
                  "chert_raypath: bad counts");
    const long long n = static_cast<long long>(n_fields) * n_rcv;
    raypath_kernel<<<(unsigned)((n + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        d_par, n_fields, n_nodes, d_src, d_rcv, n_rcv, cap, d_paths, d_len);
    return launch_check("chert_raypath");
}

extern "C" int chert_parent_ties(const void* d_Vsel, const void* d_Asel, int n_modes, int n_classes,
                                 int precision, int nx, int ny, int nz, double dx,
                                 const int32_t* d_class_of_node, const int32_t* offsets, int n_off,
                                 const int64_t* d_sources, int n_sources, const void* d_tauR,
                                 const void* d_tauI, double rel_tol, uint8_t* d_tieR, uint8_t* d_tieI,
                                 unsigned long long* d_counts, void* stream) {
    const char* who = "chert_parent_ties";
    CHERT_REQUIRE(d_Vsel && d_Asel && d_class_of_node && d_sources && d_tauR && d_tauI, "%s: NULL argument", who);
    CHERT_REQUIRE(n_modes >= 1 && n_modes <= 3 && n_classes >= 1 && n_sources >= 1, "%s: bad counts", who);
    CHERT_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1 && (long long)nx * ny * nz < (1LL << 31), "%s: bad lattice", who);
    CHERT_REQUIRE(dx > 0 && rel_tol >= 0, "%s: dx and rel_tol must be positive", who);
    CHERT_REQUIRE((long long)n_sources * n_modes <= 65535, "%s: at most 65535 fields per call", who);
    CHERT_REQUIRE(precision == CHERT_FP64 || precision == CHERT_FP32 || precision == CHERT_MIXED ||
                      precision == CHERT_FP32_ACC64, "%s: precision=%d", who, precision);
    Offsets off;
    int rc = fill_offsets(off, offsets, n_off, who);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n_fields = n_sources * n_modes;
    if (d_counts) {
        cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * n_fields * 2, s);
        if (e != cudaSuccess) return cuda_fail(e, "chert_parent_ties: memset");
    }
    const long long n = (long long)nx * ny * nz;
    const dim3 grid((unsigned)((n + 255) / 256), n_fields, 2);
    if (precision == CHERT_FP64)
        parent_ties_kernel<double, double><<<grid, 256, 0, s>>>(
            static_cast<const double*>(d_Vsel), static_cast<const double*>(d_Asel), n_modes, n_classes, off, nx, ny,
            nz, dx, d_class_of_node, d_sources, static_cast<const double*>(d_tauR),
            static_cast<const double*>(d_tauI), rel_tol, d_tieR, d_tieI, d_counts);
    else if (precision == CHERT_FP32_ACC64)
        parent_ties_kernel<float, double><<<grid, 256, 0, s>>>(
            static_cast<const float*>(d_Vsel), static_cast<const float*>(d_Asel), n_modes, n_classes, off, nx, ny,
            nz, dx, d_class_of_node, d_sources, static_cast<const double*>(d_tauR),
            static_cast<const double*>(d_tauI), rel_tol, d_tieR, d_tieI, d_counts);
    else
        parent_ties_kernel<float, float><<<grid, 256, 0, s>>>(
            static_cast<const float*>(d_Vsel), static_cast<const float*>(d_Asel), n_modes, n_classes, off, nx, ny,
            nz, dx, d_class_of_node, d_sources, static_cast<const float*>(d_tauR),
            static_cast<const float*>(d_tauI), rel_tol, d_tieR, d_tieI, d_counts);
    return launch_check(who);
}

extern "C" int chert_set_relax_points_per_thread(int ppt) {
    CHERT_REQUIRE(ppt == 0 || ppt == 1 || ppt == 2 || ppt == 4,
                  "chert_set_relax_points_per_thread: ppt=%d (0, 1, 2 or 4)", ppt);
    return g_relax_ppt.exchange(ppt);
}

extern "C" int chert_set_relax_scheduler(int scheduler) {
    if (scheduler < 0) return g_relax_sched.load();
    CHERT_REQUIRE(scheduler <= 3, "chert_set_relax_scheduler: scheduler=%d (0, 1, 2 or 3)", scheduler);
    return g_relax_sched.exchange(scheduler);
}
