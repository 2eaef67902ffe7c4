// kernels_3d.cu -- the three-dimensional split (Section 2.1): face
// coefficients in the three rotated layouts, and the line kernel's 3-D form.
//
// Layouts.  T is [nz][ny][nx] (x fastest) between steps.  The x-update reads
// lines along x indexed (z, y) and writes its result indexed (x, z, y); the
// y-update reads that as lines along y indexed (x, z) and writes (y, x, z);
// the z-update reads lines along z indexed (y, x) and writes (z, y, x).  So
// every update reads whole contiguous lines and no transpose pass is needed.
// The coefficients of each axis are stored in the layout its update reads.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "aniso_internal.h"
#include "line4_kernel.cuh"

namespace aniso {

// One thread per cell (i, j, k): the three faces i+1/2, j+1/2, k+1/2 of the
// cell.  b is averaged to the face from the two cells beside it (wrapped when
// periodic); the normal coefficient is kappa + (1 - kappa) b_d^2 and the two
// transverse ones (1 - kappa) b_d b_a, (1 - kappa) b_d b_b with (d, a, b) =
// (x, y, z), (y, z, x), (z, x, y).  Zero-flux boundary faces are zero.  FP64
// arithmetic with explicitly rounded operations (no contraction), one rounding
// to the storage type (FP64, FP32 or FP16).
template <typename B, typename C>
__global__ void face_coeffs3_kernel(const B *bx, const B *by, const B *bz, int nx, int ny, int nz, int bc,
                                    double kappa, C *cx0, C *cx1, C *cx2, C *cy0, C *cy1, C *cy2, C *cz0,
                                    C *cz1, C *cz2)
{
    const size_t cells = (size_t)nx * ny * nz;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < cells; o += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(o % nx), j = (int)((o / nx) % ny), k = (int)(o / ((size_t)nx * ny));
        const int ix[3] = {i, j, k}, n3[3] = {nx, ny, nz};
        const size_t st[3] = {1, (size_t)nx, (size_t)nx * ny};
        // destination index of the cell in the layout of each axis's update
        const size_t dst[3] = {o, ((size_t)i * nz + k) * ny + j, ((size_t)j * nx + i) * nz + k};
        C *outs[3][3] = {{cx0, cx1, cx2}, {cy0, cy1, cy2}, {cz0, cz1, cz2}};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int a = (d + 1) % 3, b = (d + 2) % 3;
            double cn = 0.0, ca = 0.0, cb = 0.0;
            if (bc != 0 || ix[d] < n3[d] - 1) {
                const int nb = ix[d] + 1 < n3[d] ? ix[d] + 1 : 0;
                const size_t o1 = o - (size_t)ix[d] * st[d] + (size_t)nb * st[d];
                const double f[3] = {__dmul_rn(0.5, __dadd_rn((double)bx[o], (double)bx[o1])),
                                     __dmul_rn(0.5, __dadd_rn((double)by[o], (double)by[o1])),
                                     __dmul_rn(0.5, __dadd_rn((double)bz[o], (double)bz[o1]))};
                const double omk = __dsub_rn(1.0, kappa);
                cn = __dadd_rn(kappa, __dmul_rn(omk, __dmul_rn(f[d], f[d])));
                ca = __dmul_rn(omk, __dmul_rn(f[d], f[a]));
                cb = __dmul_rn(omk, __dmul_rn(f[d], f[b]));
            }
            outs[d][0][dst[d]] = to_store<C>(cn);
            outs[d][1][dst[d]] = to_store<C>(ca);
            outs[d][2][dst[d]] = to_store<C>(cb);
        }
    }
}

cudaError_t launch_face_coeffs3(int prec, int coef_fp16, const void *bx, const void *by, const void *bz, int nx,
                                int ny, int nz, int bc, double kappa, void *const c[9], cudaStream_t s)
{
    const size_t cells = (size_t)nx * ny * nz;
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((cells + threads - 1) / threads, 152 * 16);
    if (coef_fp16) {
        if (prec == PREC_FP64) return cudaErrorInvalidValue;
        __half *h[9];
        for (int k = 0; k < 9; ++k) h[k] = static_cast<__half *>(c[k]);
        face_coeffs3_kernel<float, __half><<<blocks, threads, 0, s>>>(
            static_cast<const float *>(bx), static_cast<const float *>(by), static_cast<const float *>(bz), nx, ny, nz,
            bc, kappa, h[0], h[1], h[2], h[3], h[4], h[5], h[6], h[7], h[8]);
        return cudaGetLastError();
    }
    if (prec == PREC_FP64)
        face_coeffs3_kernel<double, double><<<blocks, threads, 0, s>>>(
            static_cast<const double *>(bx), static_cast<const double *>(by), static_cast<const double *>(bz), nx, ny,
            nz, bc, kappa, static_cast<double *>(c[0]), static_cast<double *>(c[1]), static_cast<double *>(c[2]),
            static_cast<double *>(c[3]), static_cast<double *>(c[4]), static_cast<double *>(c[5]),
            static_cast<double *>(c[6]), static_cast<double *>(c[7]), static_cast<double *>(c[8]));
    else
        face_coeffs3_kernel<float, float><<<blocks, threads, 0, s>>>(
            static_cast<const float *>(bx), static_cast<const float *>(by), static_cast<const float *>(bz), nx, ny, nz,
            bc, kappa, static_cast<float *>(c[0]), static_cast<float *>(c[1]), static_cast<float *>(c[2]),
            static_cast<float *>(c[3]), static_cast<float *>(c[4]), static_cast<float *>(c[5]),
            static_cast<float *>(c[6]), static_cast<float *>(c[7]), static_cast<float *>(c[8]));
    return cudaGetLastError();
}

template <typename K> static cudaError_t run4_3d(K kern, const Line2Args &a, int nblocks, int nthreads, size_t smem,
                                                 cudaStream_t s)
{
    if (smem > 47 * 1024) {  // static shared memory counts against the 48 KB default
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        if ((size_t)fa.maxDynamicSharedSizeBytes < smem &&
            (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
            return e;
    }
    kern<<<nblocks, nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_line4_3d(int prec, int coef_fp16, const Line2Args &a, int nblocks, int nthreads, size_t smem,
                            cudaStream_t s)
{
    const bool vl = a.limiter == LIM_VANLEER;
    if (coef_fp16 && prec == PREC_FP64) return cudaErrorInvalidValue;
    if (a.one.mu == 0.0 && a.one.mu2 == 0.0) {  // purely implicit update (4-step halves)
        if (prec == PREC_FP64)
            return run4_3d(line4_kernel<double, double, false, true, false, true>, a, nblocks, nthreads, smem, s);
        if (coef_fp16)
            return run4_3d(line4_kernel<float, __half, false, true, false, true>, a, nblocks, nthreads, smem, s);
        return run4_3d(line4_kernel<float, float, false, true, false, true>, a, nblocks, nthreads, smem, s);
    }
    if (coef_fp16)
        return vl ? run4_3d(line4_kernel<float, __half, true, true>, a, nblocks, nthreads, smem, s)
                  : run4_3d(line4_kernel<float, __half, false, true>, a, nblocks, nthreads, smem, s);
    if (prec == PREC_FP64)
        return vl ? run4_3d(line4_kernel<double, double, true, true>, a, nblocks, nthreads, smem, s)
                  : run4_3d(line4_kernel<double, double, false, true>, a, nblocks, nthreads, smem, s);
    return vl ? run4_3d(line4_kernel<float, float, true, true>, a, nblocks, nthreads, smem, s)
              : run4_3d(line4_kernel<float, float, false, true>, a, nblocks, nthreads, smem, s);
}

}  // namespace aniso
