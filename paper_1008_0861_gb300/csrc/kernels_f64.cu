// FP64 instantiations of the sweep kernels.
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

cudaError_t launch_line_f64(const LineArgs &a, int nblocks, int nthreads, size_t smem, cudaStream_t s)
{
    cudaError_t err = prep(line_sweep_kernel<double, double, false>, smem);
    if (err != cudaSuccess) return err;
    line_sweep_kernel<double, double, false><<<nblocks, nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_col_f64(const ColArgs &a, int nblocks, int nthreads, size_t smem, cudaStream_t s)
{
    cudaError_t err = prep(col_sweep_kernel<double, double, false>, smem);
    if (err != cudaSuccess) return err;
    col_sweep_kernel<double, double, false><<<nblocks, nthreads, smem, s>>>(a);
    return cudaGetLastError();
}


cudaError_t launch_line2_f64(const Line2Args &a, int nblocks, int nthreads, size_t smem, cudaStream_t s)
{
    cudaError_t err = prep(line2_kernel<double, double, false>, smem);
    if (err != cudaSuccess) return err;
    line2_kernel<double, double, false><<<nblocks, nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace aniso
