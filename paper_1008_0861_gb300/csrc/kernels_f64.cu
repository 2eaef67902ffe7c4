// FP64 instantiations of the sweep kernels.
#include "line3_kernel.cuh"

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

cudaError_t launch_line3_f64(const Line3Args &a, int nthreads, size_t smem, cudaStream_t s)
{
    cudaError_t err = prep(line3_kernel<double, double>, smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0, dev = 0, sms = 0;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, line3_kernel<double, double>, nthreads, smem)) !=
        cudaSuccess)
        return err;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = (per_sm > 0 ? per_sm : 1) * sms;
    if (grid > a.total_groups) grid = a.total_groups;
    line3_kernel<double, double><<<grid, nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

size_t line3_smem_f64(int n, int team, int lpb) { return (size_t)line3_plan<double, double>(n, team, lpb).bytes; }

size_t line3_stage_f64(int n, int team, int lpb) { return (size_t)line3_plan<double, double>(n, team, lpb).work; }

}  // namespace aniso
