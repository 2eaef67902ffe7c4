// FP32 instantiations of the sweep kernels (FP32 or FP16 face coefficients).
#include "line2_kernel.cuh"

namespace aniso {

// Opt in to the dynamic shared memory a launch needs (above the 48 KB
// default), never more than requested so the kernel's static shared memory
// still fits under the per-block limit.
template <typename K> static cudaError_t prep(K kern, size_t smem)
{
    if (smem <= 47 * 1024) return cudaSuccess;  // static shared memory counts too
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename K> static cudaError_t go(K kern, int nblocks, int nthreads, size_t smem, cudaStream_t s,
                                              const LineArgs &a)
{
    cudaError_t err = prep(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<nblocks, nthreads, smem, s>>>(a);
    return cudaGetLastError();
}
template <typename K> static cudaError_t goc(K kern, int nblocks, int nthreads, size_t smem, cudaStream_t s,
                                               const ColArgs &a)
{
    cudaError_t err = prep(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<nblocks, nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_line_f32(int coef_fp16, bool kahan, const LineArgs &a, int nblocks, int nthreads, size_t smem,
                            cudaStream_t s)
{
    if (coef_fp16)
        return kahan ? go(line_sweep_kernel<float, __half, true>, nblocks, nthreads, smem, s, a)
                     : go(line_sweep_kernel<float, __half, false>, nblocks, nthreads, smem, s, a);
    return kahan ? go(line_sweep_kernel<float, float, true>, nblocks, nthreads, smem, s, a)
                 : go(line_sweep_kernel<float, float, false>, nblocks, nthreads, smem, s, a);
}

cudaError_t launch_col_f32(int coef_fp16, bool kahan, const ColArgs &a, int nblocks, int nthreads, size_t smem,
                           cudaStream_t s)
{
    if (coef_fp16)
        return kahan ? goc(col_sweep_kernel<float, __half, true>, nblocks, nthreads, smem, s, a)
                     : goc(col_sweep_kernel<float, __half, false>, nblocks, nthreads, smem, s, a);
    return kahan ? goc(col_sweep_kernel<float, float, true>, nblocks, nthreads, smem, s, a)
                 : goc(col_sweep_kernel<float, float, false>, nblocks, nthreads, smem, s, a);
}

template <typename K> static cudaError_t go2(K kern, int nblocks, int nthreads, size_t smem, cudaStream_t s,
                                               const Line2Args &a)
{
    cudaError_t err = prep(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<nblocks, nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_line2_f32(int coef_fp16, const Line2Args &a, int nblocks, int nthreads, size_t smem,
                             cudaStream_t s, bool kahan)
{
    if (coef_fp16)
        return kahan ? go2(line2_kernel<float, __half, true>, nblocks, nthreads, smem, s, a)
                     : go2(line2_kernel<float, __half, false>, nblocks, nthreads, smem, s, a);
    return kahan ? go2(line2_kernel<float, float, true>, nblocks, nthreads, smem, s, a)
                 : go2(line2_kernel<float, float, false>, nblocks, nthreads, smem, s, a);
}

}  // namespace aniso
