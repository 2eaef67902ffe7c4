// Instantiations and launch configuration of the long-line kernel
// (line6_kernel.cuh): FP32 state, FP32 or FP16 face coefficients.
#include "line6_kernel.cuh"

namespace aniso {

// Lines of 2048 < n <= 4096 cells (multiples of the 16-byte vector): a team
// of P = 128 lanes (4 to 8 chunks of 4 cells a lane), `lines` (2 or 4) lines
// per block: 16-byte pieces in the transposed store with four, 8-byte ones
// with two (and then two blocks per SM).  The shared memory holds the three
// per-line arrays of line4 plus the team exchange area.
bool line6_config(int prec, int coef_fp16, int n, int *team, int *lines_per_block, int *nthreads, size_t *smem,
                  int lines)
{
    if (prec != PREC_FP32) return false;
    if (n % 4 != 0 || n <= MAX_LINE2_TRANSPOSED || n > 4096) return false;
    if (coef_fp16 && n % 8 != 0) return false;
    if (lines != 2 && lines != 4) return false;
    const int m = n / 4;
    const int P = 128;
    const int L = lines;
    const size_t sm = (size_t)L * (3 * (size_t)m * 16 + 4 * (size_t)P * sizeof(float));
    if (sm > SMEM_LIMIT - 2048) return false;
    *team = P;
    *lines_per_block = L;
    *nthreads = P * L;
    *smem = sm;
    return true;
}

template <typename K> static cudaError_t run6(K kern, const Line2Args &a, int nblocks, int nthreads, size_t smem,
                                              cudaStream_t s)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    kern<<<nblocks, nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_line6(int coef_fp16, const Line2Args &a, int nblocks, int nthreads, size_t smem, cudaStream_t s)
{
    const bool vl = a.limiter == LIM_VANLEER;
    if (coef_fp16)
        return vl ? run6(line6_kernel<__half, true>, a, nblocks, nthreads, smem, s)
                  : run6(line6_kernel<__half, false>, a, nblocks, nthreads, smem, s);
    return vl ? run6(line6_kernel<float, true>, a, nblocks, nthreads, smem, s)
              : run6(line6_kernel<float, false>, a, nblocks, nthreads, smem, s);
}

}  // namespace aniso
