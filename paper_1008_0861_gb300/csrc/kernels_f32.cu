// FP32 instantiations of the sweep kernels (FP32 or FP16 face coefficients).
#include "line2_kernel.cuh"

namespace aniso {

// Opt in to the dynamic shared memory a launch needs (above the 48 KB
// default), never more than requested so the kernel's static shared memory
// still fits under the per-block limit.
template <typename K> static cudaError_t prep(K kern, size_t smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_line_f32(int coef_fp16, const LineArgs &a, int nblocks, int nthreads, size_t smem,
                            cudaStream_t s)
{
    cudaError_t err;
    if (coef_fp16) {
        if ((err = prep(line_sweep_kernel<float, __half>, smem)) != cudaSuccess) return err;
        line_sweep_kernel<float, __half><<<nblocks, nthreads, smem, s>>>(a);
    } else {
        if ((err = prep(line_sweep_kernel<float, float>, smem)) != cudaSuccess) return err;
        line_sweep_kernel<float, float><<<nblocks, nthreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_col_f32(int coef_fp16, const ColArgs &a, int nblocks, int nthreads, size_t smem,
                           cudaStream_t s)
{
    cudaError_t err;
    if (coef_fp16) {
        if ((err = prep(col_sweep_kernel<float, __half>, smem)) != cudaSuccess) return err;
        col_sweep_kernel<float, __half><<<nblocks, nthreads, smem, s>>>(a);
    } else {
        if ((err = prep(col_sweep_kernel<float, float>, smem)) != cudaSuccess) return err;
        col_sweep_kernel<float, float><<<nblocks, nthreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}


cudaError_t launch_line2_f32(int coef_fp16, const Line2Args &a, int nblocks, int nthreads, size_t smem,
                             cudaStream_t s)
{
    cudaError_t err;
    if (coef_fp16) {
        if ((err = prep(line2_kernel<float, __half>, smem)) != cudaSuccess) return err;
        line2_kernel<float, __half><<<nblocks, nthreads, smem, s>>>(a);
    } else {
        if ((err = prep(line2_kernel<float, float>, smem)) != cudaSuccess) return err;
        line2_kernel<float, float><<<nblocks, nthreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace aniso
