// Frontier label-correcting relaxation (2D scheduler 3): the fixed point of
// Eq. 31 by pushes from the nodes whose traveltime fell in the previous
// round.  Traveltimes are non-negative, so the IEEE bit patterns of the
// values (float or double; +inf included) order like the values themselves
// and an unsigned atomicMin on them keeps the least candidate; a push that
// lowered its target marks the target for the next round.  One CTA per field
// component: the two frontier bitmaps (this round, next round) live in shared
// memory, the traveltimes in global memory (read through L2, where the
// atomics land).  When no node changed in a round, a pull pass writes the
// parents (Eq. 33, ties to the smallest node index) and confirms that no
// in-neighbour improves any node.  Same weights and the same rounded
// additions as the sweeps, so the same fixed point, bit for bit.
#pragma once
#include <stdint.h>

namespace chert {
namespace frontier {

template <typename T>
struct Bits;
template <>
struct Bits<float> {
    using U = unsigned int;
    static __device__ __forceinline__ U enc(float v) { return __float_as_uint(v); }
    static __device__ __forceinline__ float dec(U u) { return __uint_as_float(u); }
};
template <>
struct Bits<double> {
    using U = unsigned long long;
    static __device__ __forceinline__ U enc(double v) { return (U)__double_as_longlong(v); }
    static __device__ __forceinline__ double dec(U u) { return __longlong_as_double((long long)u); }
};

struct Args {
    int nx, nz, n_classes, n_modes, max_rounds;
    double dx;
    const int32_t* cls;
    const int64_t* src;
    void *tauR, *tauI;
    int32_t *parR, *parI;
    const void *Vsel, *Asel;   // [n_modes][n_classes][n_off]
    int* status;               // [field*2 + component]: rounds used, -1 = cap hit or a failed check
};

}  // namespace frontier
}  // namespace chert
