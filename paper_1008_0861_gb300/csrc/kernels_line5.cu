// Host side of the TMA-staged line kernel (line5_kernel.cuh): tensor maps,
// block shape, launches.  FP32 state and coefficients; lines of 768 to 1024
// cells that are whole 128-byte rows, one warp per line, 8 lines per block.
#include <cudaTypedefs.h>

#include <mutex>

#include "line5_kernel.cuh"

namespace aniso {

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

// The array as rows of 32 floats (128 bytes), tiles of box_rows rows, written
// to shared memory with the 128-byte swizzle.
bool make_map(CUtensorMap *m, const void *ptr, size_t floats, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || floats % 32 || ((uintptr_t)ptr & 15) || box_rows < 1 || box_rows > 256) return false;
    cuuint64_t dims[2] = {32, (cuuint64_t)(floats / 32)};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int L5_UMAX = 8;  // 4-cell chunks per lane at most: 32 lanes x 32 cells = 1024
constexpr int L5_WARPS = 8;

template <bool VL> void *kernel_ptr() { return reinterpret_cast<void *>(line5_kernel<L5_UMAX, VL, 1>); }

int grid_limit(const void *kern, int nthreads, size_t smem)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return -1;
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthreads, smem) != cudaSuccess) return -1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    return per_sm * sms;
}

}  // namespace

bool line5_available() { return encode_fn() != nullptr; }

bool line5_config(int prec, int coef_fp16, int n, int *team, int *lines_per_block, int *nthreads, size_t *stage)
{
    if (prec != PREC_FP32 || coef_fp16) return false;
    if (n % 32 != 0 || n < 768 || n > 1024) return false;
    const int m = n / 4;
    const int P = 32;
    if ((m + P - 1) / P > L5_UMAX) return false;
    const int L = L5_WARPS;  // one line per warp
    if ((n / 32) * L > 256) return false;
    *team = P;
    *lines_per_block = L;
    *nthreads = L5_WARPS * 32;
    *stage = line5_smem(n, L).total;
    return true;
}

bool line5_make_maps(Line5Job &J, const void *Tin, const void *g, const void *e, size_t cells)
{
    const int rows = J.n / 32;
    return make_map(&J.tm_T, Tin, cells, rows * J.lines_per_block) && make_map(&J.tm_T1, Tin, cells, rows) &&
           make_map(&J.tm_g, g, cells, rows * J.lines_per_block) &&
           make_map(&J.tm_e, e, cells, rows * J.lines_per_block);
}

int line5_prepare(int limiter, int nthreads, size_t stage)
{
    const void *kern = limiter == LIM_VANLEER ? kernel_ptr<true>() : kernel_ptr<false>();
    return grid_limit(kern, nthreads, stage + 1024);
}

// One block per tile (grid = all tiles).  Launch attributes were set by
// line5_prepare, outside any stream capture.
cudaError_t launch_line5(const Line5Args &a0, int nthreads, size_t stage, cudaStream_t s)
{
    Line5Args a = a0;
    const size_t smem = stage + 1024;
    if (a.wait_limit == 0) a.wait_limit = 1u << 20;
    if (a.limiter == LIM_VANLEER) line5_kernel<L5_UMAX, true, 1><<<a.total_tiles, nthreads, smem, s>>>(a, (unsigned)stage);
    else line5_kernel<L5_UMAX, false, 1><<<a.total_tiles, nthreads, smem, s>>>(a, (unsigned)stage);
    return cudaGetLastError();
}

}  // namespace aniso
