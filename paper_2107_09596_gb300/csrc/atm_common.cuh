// atm_common.cuh -- error reporting shared by the library's translation units.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <string>

#include <cuda_runtime.h>

#include "../../include/atm.h"

namespace atm {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
inline std::string &last_error()
{
    static thread_local std::string s;
    return s;
}

inline atm_status fail(atm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    last_error() = buf;
    return st;
}

#define ATM_CK(call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::atm::fail(ATM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define ATM_TRY(expr)                         \
    do {                                      \
        atm_status s_ = (expr);               \
        if (s_ != ATM_OK) return s_;          \
    } while (0)

}  // namespace atm
