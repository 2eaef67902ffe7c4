// Instantiations of the warp-per-line kernel and of the explicit step (FP32
// with FP32 or FP16 face coefficients, FP64), one variant per limiter family.
#include "explicit_kernel.cuh"

namespace aniso {

template <typename K> static cudaError_t run4(K kern, const Line2Args &a, int nblocks, int nthreads, size_t smem,
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

cudaError_t launch_line4(int prec, int coef_fp16, const Line2Args &a, int nblocks, int nthreads, size_t smem,
                         cudaStream_t s)
{
    const bool vl = a.limiter == LIM_VANLEER;
    if (!a.jobs && a.one.mu == 0.0 && a.one.chi_alpha == 0.0) {  // purely implicit update (4-step halves)
        if (prec == PREC_FP64)
            return run4(line4_kernel<double, double, false, false, false, true>, a, nblocks, nthreads, smem, s);
        if (coef_fp16)
            return run4(line4_kernel<float, __half, false, false, false, true>, a, nblocks, nthreads, smem, s);
        return run4(line4_kernel<float, float, false, false, false, true>, a, nblocks, nthreads, smem, s);
    }
    if (!a.jobs && a.one.chi_alpha != 0.0) {  // temperature-dependent diffusivity (single grids)
        if (coef_fp16) return cudaErrorInvalidValue;
        if (prec == PREC_FP64)
            return vl ? run4(line4_kernel<double, double, true, false, true>, a, nblocks, nthreads, smem, s)
                      : run4(line4_kernel<double, double, false, false, true>, a, nblocks, nthreads, smem, s);
        return vl ? run4(line4_kernel<float, float, true, false, true>, a, nblocks, nthreads, smem, s)
                  : run4(line4_kernel<float, float, false, false, true>, a, nblocks, nthreads, smem, s);
    }
    if (a.tmem && prec == PREC_FP32) {  // gamma in tensor memory
        if (coef_fp16)
            return vl ? run4(line4_kernel<float, __half, true, false, false, false, true>, a, nblocks, nthreads, smem, s)
                      : run4(line4_kernel<float, __half, false, false, false, false, true>, a, nblocks, nthreads, smem, s);
        return vl ? run4(line4_kernel<float, float, true, false, false, false, true>, a, nblocks, nthreads, smem, s)
                  : run4(line4_kernel<float, float, false, false, false, false, true>, a, nblocks, nthreads, smem, s);
    }
    if (prec == PREC_FP64)
        return vl ? run4(line4_kernel<double, double, true>, a, nblocks, nthreads, smem, s)
                  : run4(line4_kernel<double, double, false>, a, nblocks, nthreads, smem, s);
    if (coef_fp16)
        return vl ? run4(line4_kernel<float, __half, true>, a, nblocks, nthreads, smem, s)
                  : run4(line4_kernel<float, __half, false>, a, nblocks, nthreads, smem, s);
    return vl ? run4(line4_kernel<float, float, true>, a, nblocks, nthreads, smem, s)
              : run4(line4_kernel<float, float, false>, a, nblocks, nthreads, smem, s);
}

template <typename K> static int occ4(K kern, int nthreads, size_t smem)
{
    if (smem > 47 * 1024) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return -1;
        if ((size_t)fa.maxDynamicSharedSizeBytes < smem &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -1;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, nthreads, smem) != cudaSuccess) return -1;
    return blocks;
}

int line4_tm_cols(int n, int team)
{
    const int m = n / 4, U = m / team, V = U + (m % team ? 1 : 0);
    return 8 * V <= 32 ? 32 : 64;
}

// The kernel keeps 16-byte chunk c of a line at c ^ ((c >> s) & 7) inside
// its group of 8 chunks (the last, incomplete group unswizzled).  The
// coalesced phases have the 8 lanes of a quarter warp touch one whole group,
// conflict-free under any such permutation.  The segment phases have lane t
// walk chunks c_lo(t) + u of its segment (U + 1 chunks for the first m mod P
// lanes, U for the rest), so a quarter warp's chunks lie a segment length
// apart and their bank groups (chunk mod 8) repeat unless the shift spreads
// them.  Each candidate (log2 U, none, 1..6) is scored by the wavefronts of
// those walks, the largest number of a quarter's lanes on one bank group,
// summed over the steps u and the quarters; the first lowest wins.
int line4_swizzle(int prec, int n, int team)
{
    const int N = prec == PREC_FP64 ? 2 : 4;
    const int m = n / N, P = team;
    if (P < 8 || m < 8) return 0;  // a quarter warp spans several lines
    const int U = m / P, rr = m % P, V = U + (rr ? 1 : 0);
    const int mfull = m & ~7;
    int logU = 0;
    while ((2 << logU) <= U) ++logU;
    int best = 0;
    long best_w = -1;
    for (int code = 0; code <= 7; ++code) {
        const int sh = code >= 2 ? code - 1 : logU, msk = code == 1 ? 0 : 7;
        long w = 0;
        for (int u = 0; u < V; ++u)
            for (int q0 = 0; q0 < P; q0 += 8) {
                int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int t = q0; t < q0 + 8; ++t) {
                    if (u >= U + (t < rr ? 1 : 0)) continue;
                    const int c = t * U + (t < rr ? t : rr) + u;
                    ++cnt[(c < mfull ? c ^ ((c >> sh) & msk) : c) & 7];
                }
                int mx = 0;
                for (int g = 0; g < 8; ++g) mx = cnt[g] > mx ? cnt[g] : mx;
                w += mx;
            }
        if (best_w < 0 || w < best_w) {
            best_w = w;
            best = code;
        }
    }
    return best;
}

int line4_blocks_per_sm(int prec, int coef_fp16, int limiter, int nthreads, size_t smem, bool tmem, int tm_cols)
{
    const bool vl = limiter == LIM_VANLEER;
    if (tmem && prec == PREC_FP32) {
        // CUDA's occupancy calculator answers 1 for a kernel that allocates
        // tensor memory, while 5-7 such blocks were measured resident.  The
        // shared-memory form has the same registers and static shared memory:
        // its answer at this dynamic size, capped by the TMEM columns (at
        // most 448 of an SM's 512 were found in use at once: seven 64-column
        // blocks where eight fit otherwise).
        const int cap = 448 / (tm_cols > 0 ? tm_cols : 64);
        const int occ = line4_blocks_per_sm(prec, coef_fp16, limiter, nthreads, smem, false);
        return occ < cap ? occ : cap;
    }
    if (prec == PREC_FP64)
        return vl ? occ4(line4_kernel<double, double, true>, nthreads, smem)
                  : occ4(line4_kernel<double, double, false>, nthreads, smem);
    if (coef_fp16)
        return vl ? occ4(line4_kernel<float, __half, true>, nthreads, smem)
                  : occ4(line4_kernel<float, __half, false>, nthreads, smem);
    return vl ? occ4(line4_kernel<float, float, true>, nthreads, smem)
              : occ4(line4_kernel<float, float, false>, nthreads, smem);
}

template <typename K> static cudaError_t run_explicit(K kern, const ExpArgs &a, cudaStream_t s)
{
    const int rows_total = (a.ny + a.rows - 1) / a.rows;
    const dim3 block(32, 8), grid((a.nx + 31) / 32, (rows_total + 7) / 8);
    kern<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_explicit(int prec, int coef_fp16, const ExpArgs &a, cudaStream_t s)
{
    const bool vl = a.limiter == LIM_VANLEER;
    if (prec == PREC_FP64)
        return vl ? run_explicit(explicit_kernel<double, double, true>, a, s)
                  : run_explicit(explicit_kernel<double, double, false>, a, s);
    if (coef_fp16)
        return vl ? run_explicit(explicit_kernel<float, __half, true>, a, s)
                  : run_explicit(explicit_kernel<float, __half, false>, a, s);
    return vl ? run_explicit(explicit_kernel<float, float, true>, a, s)
              : run_explicit(explicit_kernel<float, float, false>, a, s);
}

}  // namespace aniso
