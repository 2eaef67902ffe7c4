// Launch configuration, face coefficients, transposes and FP64 totals.
#include "sweep_kernels.cuh"

namespace aniso {

cudaError_t launch_line_f32(int coef_fp16, bool kahan, const LineArgs &a, int nblocks, int nthreads, size_t smem,
                            cudaStream_t s);
cudaError_t launch_col_f32(int coef_fp16, bool kahan, const ColArgs &a, int nblocks, int nthreads, size_t smem,
                           cudaStream_t s);
cudaError_t launch_line_f64(const LineArgs &a, int nblocks, int nthreads, size_t smem, cudaStream_t s);
cudaError_t launch_col_f64(const ColArgs &a, int nblocks, int nthreads, size_t smem, cudaStream_t s);
cudaError_t launch_line2_f32(int coef_fp16, const Line2Args &a, int nblocks, int nthreads, size_t smem,
                             cudaStream_t s, bool kahan);
cudaError_t launch_line2_f64(const Line2Args &a, int nblocks, int nthreads, size_t smem, cudaStream_t s);
static int pow2floor(int v)
{
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}
static int pow2ceil(int v)
{
    int p = 1;
    while (p < v) p *= 2;
    return p;
}
static size_t esize(int prec) { return prec == PREC_FP64 ? 8 : 4; }

// Target: about 32 cells per thread, one warp per line up to 1024 cells,
// at most 512 threads per line; ~110 KB of shared memory per block so that
// two blocks fit on an SM when the line allows it.
void line_config(int prec, int n, int *team, int *lines_per_block, int *nthreads)
{
    int P;
    if (n < 32) P = pow2floor(n);
    else {
        P = pow2ceil((n + 31) / 32);
        if (P < 32) P = 32;
        if (P > 512) P = 512;
    }
    int lpb = P >= 256 ? 1 : 256 / P;
    const size_t per_line = line_smem_bytes(prec, n, P, 1);
    while (lpb > 1 && per_line * lpb > 110 * 1024) lpb /= 2;
    *team = P;
    *lines_per_block = lpb;
    *nthreads = P * lpb;
}

size_t line_smem_bytes(int prec, int n, int team, int lines_per_block)
{
    const size_t np = (size_t)n + (n >> 5) + 1;
    return (size_t)lines_per_block * (3 * np + 8 * (size_t)team) * esize(prec);
}

void col_config(int prec, int ny, int *P_out, int *Wb_out, int *nthreads)
{
    const int wmin = prec == PREC_FP64 ? 8 : 16;  // 64-byte row segments at least
    int NT = prec == PREC_FP64 ? 256 : 512;
    int P = 1, Wb = NT;
    for (;;) {
        P = pow2floor(ny / 16 > 0 ? ny / 16 : 1);
        if (P > NT / wmin) P = NT / wmin;
        if (P > ny) P = pow2floor(ny);
        Wb = NT / P;
        if (col_smem_bytes(prec, ny, P, Wb) <= 113 * 1024 || Wb <= wmin || NT <= 128) break;
        NT /= 2;
    }
    *P_out = P;
    *Wb_out = Wb;
    *nthreads = NT;
}

size_t col_smem_bytes(int prec, int ny, int P, int Wb)
{
    return (3 * ((size_t)ny + P) * Wb + 8 * (size_t)P * Wb) * esize(prec);
}

cudaError_t launch_line(int prec, int coef_fp16, const LineArgs &a, int nblocks, int nthreads,
                        size_t smem, cudaStream_t s, bool kahan)
{
    if (prec == PREC_FP64) return launch_line_f64(a, nblocks, nthreads, smem, s);
    return launch_line_f32(coef_fp16, kahan, a, nblocks, nthreads, smem, s);
}

cudaError_t launch_col(int prec, int coef_fp16, const ColArgs &a, int nblocks, int nthreads,
                       size_t smem, cudaStream_t s, bool kahan)
{
    if (prec == PREC_FP64) return launch_col_f64(a, nblocks, nthreads, smem, s);
    return launch_col_f32(coef_fp16, kahan, a, nblocks, nthreads, smem, s);
}

size_t line2_smem_bytes(int prec, int n, int team, int lines_per_block)
{
    const int N = prec == PREC_FP64 ? 2 : 4;
    size_t words = (size_t)lines_per_block * (3 * (size_t)n + N);
    if (team > 32) words += (size_t)lines_per_block * 8 * team;
    return words * esize(prec);
}

// About 4 chunks (16 FP32 / 8 FP64 cells) per segment, so that a 256-thread
// block needs ~49 KB of shared memory and four blocks share an SM; 256
// threads per block unless a line needs more; the segment grows when shared
// memory is short.
bool line2_config(int prec, int n, bool transposed, int *team, int *lines_per_block, int *nthreads,
                  size_t *smem, int seg_chunks)
{
    const int sc = seg_chunks > 0 ? seg_chunks : 4;
    const int N = prec == PREC_FP64 ? 2 : 4;
    if (n % N != 0 || n < 2 * N) return false;
    if (transposed && n > MAX_LINE2_TRANSPOSED) return false;
    const int m = n / N;
    int P = pow2ceil((m + sc - 1) / sc);
    if (P > m) P = pow2floor(m);
    if (P > 512) P = 512;
    for (;;) {
        const int NT = P > 256 ? P : 256;
        const int lpb = NT / P;
        const size_t sm = line2_smem_bytes(prec, n, P, lpb);
        if (sm <= SMEM_LIMIT - 1024 && (!transposed || (lpb % N == 0))) {
            *team = P;
            *lines_per_block = lpb;
            *nthreads = NT;
            *smem = sm;
            return true;
        }
        if (P == 1) return false;
        P /= 2;
    }
}

// Warp-autonomous line kernel: a team of P <= 32 lanes per line with about
// seg_chunks (default 4: 16 FP32 / 8 FP64 cells) chunks per lane or more, at
// most 16 chunks a lane; the warp's shared area holds 3 arrays of its lines' chunks.  Blocks
// of `warps` warps (default 4); with a transposed output the block's line
// count must fill whole 16-byte stores.
bool line4_config(int prec, int n, bool transposed, int warps, int seg_chunks, int *team, int *lines_per_block,
                  int *nthreads, size_t *smem, bool tmem)
{
    const int N = prec == PREC_FP64 ? 2 : 4;
    if (n % N != 0 || n < 2 * N) return false;
    if (transposed && n > MAX_LINE2_TRANSPOSED) return false;
    const int m = n / N, sc = seg_chunks > 0 ? seg_chunks : 4;
    int P = pow2floor(m / sc > 0 ? m / sc : 1);
    if (P > 32) P = 32;
    const int U = m / P, V = U + (m % P ? 1 : 0);
    if (V > 16) return false;
    int NW = warps > 0 ? warps : 4;
    if (NW > 8) NW = 8;
    const int L = 32 / P;
    while (transposed && (NW * L) % N != 0) NW *= 2;
    if (NW > 8) return false;
    // the tensor-memory form: each lane keeps 4 V columns of gamma and 4 V of
    // T_old, of the block's 64
    if (tmem && (prec != PREC_FP32 || NW != 4 || 8 * V > 64)) return false;
    const int narr = tmem ? 2 : 3;
    const size_t sm = (size_t)NW * (narr * L * m + (N == 4 ? line4_area_pad(P, narr, m) : 0)) * 16;
    if (sm > SMEM_LIMIT - 1024) return false;
    *team = P;
    *lines_per_block = NW * L;
    *nthreads = NW * 32;
    *smem = sm;
    return true;
}

// Diagnostics of one batched line4 launch: job j's blocks are
// [block0, block0 + nblocks).  One warp per job: lane l adds the partials of
// blocks block0 + l, + 32, ... in order, then the lanes' sums are combined by
// a fixed shuffle tree, so the result does not depend on timing.
__global__ void diag_finish_kernel(const Line2Job *jobs, int njobs, const DiagPart *part, double *ring)
{
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < njobs; j += (gridDim.x * blockDim.x) >> 5) {
        const Line2Job &J = jobs[j];
        if (J.diag_slot < 0) continue;
        double sum = 0.0, mn = INFINITY, mx = -INFINITY;
        for (int b = J.block0 + lane; b < J.block0 + J.nblocks; b += 32) {
            sum += part[b].sum;
            mn = fmin(mn, part[b].mn);
            mx = fmax(mx, part[b].mx);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(full, sum, o);
            mn = fmin(mn, __shfl_xor_sync(full, mn, o));
            mx = fmax(mx, __shfl_xor_sync(full, mx, o));
        }
        if (lane == 0) {
            double *out = ring + 3 * (size_t)J.diag_slot;
            out[0] = sum;
            out[1] = mn;
            out[2] = mx;
        }
    }
}

cudaError_t launch_diag_finish(const Line2Job *jobs, int njobs, const DiagPart *part, double *ring, cudaStream_t s)
{
    if (njobs <= 0) return cudaSuccess;
    const int warps = 8;  // jobs per block
    diag_finish_kernel<<<(njobs + warps - 1) / warps, 32 * warps, 0, s>>>(jobs, njobs, part, ring);
    return cudaGetLastError();
}

__global__ void fill_nan_kernel(double *p, size_t n)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        p[k] = __longlong_as_double(0x7ff8000000000000ll);
}

cudaError_t launch_fill_nan(double *ring, size_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 4);
    fill_nan_kernel<<<blocks, 256, 0, s>>>(ring, count);
    return cudaGetLastError();
}

// Source stage of a step: T += dt Q, elementwise.
template <typename R> __global__ void source_kernel(R *T, const R *Q, R dt, size_t n)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        T[k] += dt * Q[k];
}

cudaError_t launch_source(int prec, void *T, const void *Q, double dt, size_t n, cudaStream_t s)
{
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((n + threads - 1) / threads, 152 * 8);
    if (prec == PREC_FP64)
        source_kernel<double><<<blocks, threads, 0, s>>>(static_cast<double *>(T), static_cast<const double *>(Q), dt, n);
    else
        source_kernel<float><<<blocks, threads, 0, s>>>(static_cast<float *>(T), static_cast<const float *>(Q), (float)dt, n);
    return cudaGetLastError();
}

cudaError_t launch_line2(int prec, int coef_fp16, const Line2Args &a, int nblocks, int nthreads,
                         size_t smem, cudaStream_t s, bool kahan)
{
    if (prec == PREC_FP64) return launch_line2_f64(a, nblocks, nthreads, smem, s);
    return launch_line2_f32(coef_fp16, a, nblocks, nthreads, smem, s, kahan);
}

template <typename B, typename C>
static void face_launch(const void *bx, const void *by, int nx, int ny, int bc, double kappa, void *cxx,
                        void *cxy, void *cyy, void *cyx, void *cyyT, void *cyxT, cudaStream_t s)
{
    dim3 block(256), grid((nx + 255) / 256, ny);
    face_coeffs_kernel<B, C><<<grid, block, 0, s>>>(
        static_cast<const B *>(bx), static_cast<const B *>(by), nx, ny, bc, kappa, static_cast<C *>(cxx),
        static_cast<C *>(cxy), static_cast<C *>(cyy), static_cast<C *>(cyx), static_cast<C *>(cyyT),
        static_cast<C *>(cyxT));
}

cudaError_t launch_face_coeffs(int bprec, int coef, const void *bx, const void *by, int nx, int ny,
                               int bc, double kappa, void *cxx, void *cxy, void *cyy, void *cyx,
                               void *cyyT, void *cyxT, cudaStream_t s)
{
    if (bprec == PREC_FP64) {
        if (coef == 0) face_launch<double, double>(bx, by, nx, ny, bc, kappa, cxx, cxy, cyy, cyx, cyyT, cyxT, s);
        else if (coef == 1) face_launch<double, float>(bx, by, nx, ny, bc, kappa, cxx, cxy, cyy, cyx, cyyT, cyxT, s);
        else face_launch<double, __half>(bx, by, nx, ny, bc, kappa, cxx, cxy, cyy, cyx, cyyT, cyxT, s);
    } else {
        if (coef == 0) face_launch<float, double>(bx, by, nx, ny, bc, kappa, cxx, cxy, cyy, cyx, cyyT, cyxT, s);
        else if (coef == 1) face_launch<float, float>(bx, by, nx, ny, bc, kappa, cxx, cxy, cyy, cyx, cyyT, cyxT, s);
        else face_launch<float, __half>(bx, by, nx, ny, bc, kappa, cxx, cxy, cyy, cyx, cyyT, cyxT, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_transpose(int elem_bytes, const void *in, void *out, int rows, int cols,
                             cudaStream_t s)
{
    dim3 block(32, 8), grid((cols + 31) / 32, (rows + 31) / 32);
    if (elem_bytes == 8)
        transpose_kernel<double><<<grid, block, 0, s>>>(static_cast<const double *>(in),
                                                        static_cast<double *>(out), rows, cols);
    else
        transpose_kernel<float><<<grid, block, 0, s>>>(static_cast<const float *>(in),
                                                       static_cast<float *>(out), rows, cols);
    return cudaGetLastError();
}

cudaError_t launch_totals(int prec, const void *T, size_t n, double *partials, double *result,
                          cudaStream_t s, const void *Tlo)
{
    if (prec == PREC_FP64)
        totals_partial_kernel<double><<<TOTALS_BLOCKS, 256, 0, s>>>(static_cast<const double *>(T), nullptr, n,
                                                                    partials);
    else
        totals_partial_kernel<float><<<TOTALS_BLOCKS, 256, 0, s>>>(static_cast<const float *>(T),
                                                                   static_cast<const float *>(Tlo), n, partials);
    totals_final_kernel<<<1, 32, 0, s>>>(partials, TOTALS_BLOCKS, result);
    return cudaGetLastError();
}

}  // namespace aniso
