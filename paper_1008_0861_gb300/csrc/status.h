// status.h -- host-side status helpers of the C ABI: every failing call
// records a formatted message (read back through aniso_last_error(), per host
// thread) and returns its ANISO_ERR_* code; nothing aborts or traps.
#pragma once
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/aniso.h"

namespace aniso {
void record_error(const char *msg);  // defined in aniso_api.cu
}

static inline int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    aniso::record_error(buf);
    return code;
}

// Return ANISO_ERR_OOM / ANISO_ERR_CUDA from the enclosing function when a
// CUDA runtime call fails.
#define CU(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? ANISO_ERR_OOM : ANISO_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)
