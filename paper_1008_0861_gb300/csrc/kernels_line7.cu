// Instantiations and launch configuration of the cluster line kernel
// (line7_kernel.cuh): FP32 state, plain (gamma in shared or tensor memory) or
// compensated (shared memory), FP32 or FP16 face coefficients.
#include "line7_kernel.cuh"

namespace aniso {

// n = CS * np with np = 2048 (or 1024 when n is not a multiple of 2048) and
// CS = 1, 2, 4 or 8 blocks a cluster; four lines a block.
bool line7_config(int prec, int coef_fp16, int n, int *cs, int *nthreads, size_t *smem, bool tmem)
{
    if (prec != PREC_FP32 || n <= 0) return false;
    (void)coef_fp16;
    int np = 2048;
    if (n % np != 0) np = 1024;
    if (n % np != 0) return false;
    const int c = n / np;
    if (c != 1 && c != 2 && c != 4 && c != 8) return false;
    *cs = c;
    *nthreads = L7_THREADS;
    *smem = (size_t)L7_LPB * (tmem ? 2 : 3) * (size_t)(np / 4) * 16;
    return true;
}

template <typename Kern>
static cudaError_t run7(Kern kern, const Line2Args &a, int cs, size_t smem, cudaStream_t s)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    const int groups = (a.one.nlines + L7_LPB - 1) / L7_LPB;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(groups * cs), 1, 1);
    cfg.blockDim = dim3(L7_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <bool K, bool TM, bool TO>
static cudaError_t launch7k(int coef_fp16, const Line2Args &a, int cs, size_t smem, cudaStream_t s)
{
    const bool vl = a.limiter == LIM_VANLEER;
    if (coef_fp16)
        return vl ? run7(line7_kernel<__half, true, K, TM, TO>, a, cs, smem, s)
                  : run7(line7_kernel<__half, false, K, TM, TO>, a, cs, smem, s);
    return vl ? run7(line7_kernel<float, true, K, TM, TO>, a, cs, smem, s)
              : run7(line7_kernel<float, false, K, TM, TO>, a, cs, smem, s);
}

cudaError_t launch_line7(int coef_fp16, const Line2Args &a, int cs, size_t smem, cudaStream_t s)
{
    if (a.jobs || a.one.n % cs != 0) return cudaErrorInvalidValue;
    const bool k = a.one.TinLo != nullptr;
    if (k && (!a.one.ToutLo)) return cudaErrorInvalidValue;
    // with args.tmem: the plain state keeps gamma and T_old in tensor memory
    // (two shared arrays, three blocks an SM); the compensated state keeps
    // T_old's hi and lo there (three shared arrays, two blocks an SM)
    if (k)
        return a.tmem ? launch7k<true, false, true>(coef_fp16, a, cs, smem, s)
                      : launch7k<true, false, false>(coef_fp16, a, cs, smem, s);
    return a.tmem ? launch7k<false, true, true>(coef_fp16, a, cs, smem, s)
                  : launch7k<false, false, false>(coef_fp16, a, cs, smem, s);
}

}  // namespace aniso
