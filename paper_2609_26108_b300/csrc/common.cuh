// Shared host-side helpers of libchert: error reporting and launch checks.
#pragma once
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include "chert.h"

namespace chert {

// Per-thread message of the last error (returned by chert_last_error).
void set_error(const char* fmt, ...);

inline int cuda_fail(cudaError_t e, const char* where) {
    set_error("%s: %s", where, cudaGetErrorString(e));
    return CHERT_ECUDA;
}

inline int launch_check(const char* where) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CHERT_OK : cuda_fail(e, where);
}

}  // namespace chert

#define CHERT_REQUIRE(cond, ...)                 \
    do {                                         \
        if (!(cond)) {                           \
            chert::set_error(__VA_ARGS__);       \
            return CHERT_EINVAL;                 \
        }                                        \
    } while (0)
