// noalloc.cu -- aniso_step_noalloc: a step entry point that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator, a host that has fixed its device
// memory budget before it calls us, or a plugin that must not change the
// process's allocation state.  aniso_step does allocate (its handle owns the
// face coefficients and the intermediate T* of each step), so this entry point
// keeps all of its working memory in one file-scope device array instead:
//
//   g_noalloc_scratch: NOALLOC_SCRATCH_BYTES (20 MiB + 256 bytes), allocated
//   by the CUDA runtime on first use per device (with lazy module loading,
//   when the library's module is first loaded there) and then held by that
//   GPU until the process exits.
//
// Layout of the array for a call with `cells` = nx*ny cells of `es` bytes:
//   [0, 256)                 : non-finite flag (cleared at the start of each call)
//   [256 + k*cells*es, ...)  : k = 0 T*, 1 cxx, 2 cxy, 3 cyy, 4 cyx
// so a call needs 5 * cells * es bytes: at most 1,048,576 cells in FP32 and
// 524,288 cells in FP64.
//
// All calls share the array: each call overwrites what the previous one left
// there, so two calls whose GPU work overlaps (different streams, different
// host threads) race on it and corrupt each other's results.  Serialise them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "../../include/aniso.h"
#include "aniso_internal.h"

using namespace aniso;

namespace {

constexpr size_t NOALLOC_FIELD_BYTES = 20u << 20;
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_FIELD_BYTES + 256;

// The scratch array.  In host code its name is only a stand-in for the
// device symbol; the kernels get the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void *g_scratch_ptr[MAX_DEVICES] = {nullptr};

int noalloc_fail(int code, const char *msg)
{
    record_error(msg);  // readable through aniso_last_error()
    return code;
}

// Device address of the scratch array on the current device.  Outside a
// stream capture it is looked up again on every call (with the device
// current), so a cudaDeviceReset, after which the module is loaded afresh and
// the array may sit elsewhere, never leaves a stale address behind.  Inside a
// capture only the address of the last uncaptured call on this device is
// used: the lookup itself may load the module, which a capture does not allow.
int scratch_address(cudaStream_t s, void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(ANISO_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return noalloc_fail(ANISO_ERR_UNSUPPORTED, "device index out of range");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        (void)cudaGetLastError();  // the query's own error is not sticky; treat as capturing
        cs = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return noalloc_fail(ANISO_ERR_CUDA, cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    } else if (!g_scratch_ptr[dev]) {
        return noalloc_fail(ANISO_ERR_STATE,
                            "aniso_step_noalloc: the first call on a device must come before any stream capture");
    }
    *out = g_scratch_ptr[dev];
    return ANISO_OK;
}

}  // namespace

extern "C" int aniso_step_noalloc(int nx, int ny, double dx, double dy, double chi_par, double chi_perp,
                                  int bc, int precision, const void *bx, const void *by, void *T,
                                  double dt, int nsteps, void *stream)
{
    if (nx < 3 || ny < 3) return noalloc_fail(ANISO_ERR_ARG, "aniso_step_noalloc: nx and ny must be >= 3");
    if (!(dx > 0) || !(dy > 0) || !(chi_par > 0) || !(chi_perp >= 0) || chi_perp > chi_par || !(dt > 0))
        return noalloc_fail(ANISO_ERR_ARG, "aniso_step_noalloc: need dx, dy, chi_par, dt > 0 and 0 <= chi_perp <= chi_par");
    if (bc != ANISO_BC_ZEROFLUX && bc != ANISO_BC_PERIODIC)
        return noalloc_fail(ANISO_ERR_ARG, "aniso_step_noalloc: unknown boundary condition");
    if (precision != ANISO_PREC_FP64 && precision != ANISO_PREC_FP32)
        return noalloc_fail(ANISO_ERR_ARG, "aniso_step_noalloc: unknown precision");
    if (!bx || !by || !T || nsteps < 0) return noalloc_fail(ANISO_ERR_ARG, "aniso_step_noalloc: null pointer or negative nsteps");
    const size_t es = precision == ANISO_PREC_FP64 ? 8 : 4;
    const size_t cells = (size_t)nx * (size_t)ny;
    if (5 * cells * es > NOALLOC_FIELD_BYTES) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "aniso_step_noalloc: %dx%d needs %zu bytes of scratch, above the fixed %zu "
                 "(at most %zu cells in this precision)",
                 nx, ny, 5 * cells * es, NOALLOC_FIELD_BYTES, NOALLOC_FIELD_BYTES / (5 * es));
        return noalloc_fail(ANISO_ERR_ARG, buf);
    }
    const int maxline = precision == ANISO_PREC_FP64 ? MAX_LINE_FP64 : MAX_LINE_FP32;
    if (ny > MAX_COL || nx > maxline)
        return noalloc_fail(ANISO_ERR_UNSUPPORTED, "aniso_step_noalloc: needs ny <= 1024 and nx within the line limit");
    if (nsteps == 0) return ANISO_OK;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *base = nullptr;
    int rc = scratch_address(s, &base);
    if (rc) return rc;
    unsigned char *b = static_cast<unsigned char *>(base);
    unsigned *err = reinterpret_cast<unsigned *>(b);
    void *tstar = b + 256;
    void *cxx = b + 256 + 1 * cells * es, *cxy = b + 256 + 2 * cells * es;
    void *cyy = b + 256 + 3 * cells * es, *cyx = b + 256 + 4 * cells * es;

    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return noalloc_fail(ANISO_ERR_CUDA, cudaGetErrorString(e));
    e = launch_face_coeffs(precision, precision == ANISO_PREC_FP64 ? 0 : 1, bx, by, nx, ny, bc,
                           chi_perp / chi_par, cxx, cxy, cyy, cyx, nullptr, nullptr, s);
    if (e != cudaSuccess) return noalloc_fail(ANISO_ERR_CUDA, cudaGetErrorString(e));

    const int per = bc == ANISO_BC_PERIODIC;
    const double lamx = chi_par * dt / (dx * dx), lamy = chi_par * dt / (dy * dy), mu = chi_par * dt / (dx * dy);
    LineArgs la{};
    la.limiter = LIM_VANLEER;
    la.err = err;
    la.njobs = 1;
    LineJob &X = la.one;
    X.Tin = T;
    X.Tout = tstar;
    X.g = cxx;
    X.e = cxy;
    X.lam = lamx;
    X.mu = mu;
    X.n = nx;
    X.nlines = ny;
    X.per_line = per;
    X.per_cross = per;
    int xthreads;
    line_config(precision, nx, &X.team, &X.lines_per_block, &xthreads);
    X.nblocks = (ny + X.lines_per_block - 1) / X.lines_per_block;
    const size_t xsmem = line_smem_bytes(precision, nx, X.team, X.lines_per_block);

    ColArgs ca{};
    ca.limiter = LIM_VANLEER;
    ca.err = err;
    ca.njobs = 1;
    ColJob &Y = ca.one;
    Y.Tin = tstar;
    Y.Tout = T;
    Y.g = cyy;
    Y.e = cyx;
    Y.lam = lamy;
    Y.mu = mu;
    Y.nx = nx;
    Y.ny = ny;
    Y.per_x = per;
    Y.per_y = per;
    int ythreads;
    col_config(precision, ny, &Y.P, &Y.Wb, &ythreads);
    Y.nblocks = (nx + Y.Wb - 1) / Y.Wb;
    const size_t ysmem = col_smem_bytes(precision, ny, Y.P, Y.Wb);

    // Eq. op_2step: x-update into T* (scratch), then y-update back into T.
    for (int k = 0; k < nsteps; ++k) {
        e = launch_line(precision, 0, la, X.nblocks, xthreads, xsmem, s);
        if (e != cudaSuccess) return noalloc_fail(ANISO_ERR_CUDA, cudaGetErrorString(e));
        e = launch_col(precision, 0, ca, Y.nblocks, ythreads, ysmem, s);
        if (e != cudaSuccess) return noalloc_fail(ANISO_ERR_CUDA, cudaGetErrorString(e));
    }
    return ANISO_OK;
}
