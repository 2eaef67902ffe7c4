// aniso_internal.h -- job descriptors and launch entry points shared by the
// library's translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace aniso {

enum { LIM_VANLEER = 0, LIM_ARITH = 1, LIM_MINMOD = 2, LIM_MC = 3 };
enum { PREC_FP64 = 0, PREC_FP32 = 1 };

// Longest line a block can hold on chip, per precision (three buffers of the
// line's length in shared memory).
constexpr int MAX_LINE_FP32 = 16384;
constexpr int MAX_LINE_FP64 = 8192;
// Longest column the column kernel holds on chip (3 x (ny + P) x 64 bytes).
constexpr int MAX_COL = 1024;
constexpr size_t SMEM_LIMIT = 227 * 1024;

// One contiguous-line update (Eq. xup on rows, or Eq. yup on a transposed
// grid): `nlines` lines of `n` cells, line-major.  Lines are solved by teams
// of `team` threads, `lines_per_block` teams per block.
struct LineJob {
    const void *Tin;
    void *Tout;
    const void *TinLo;  // compensated (Kahan) low parts, or nullptr
    void *ToutLo;
    const void *g;   // normal (implicit) face coefficient, face p+1/2 of each line at index p
    const void *e;   // transverse face coefficient, same layout
    double lam, mu;  // chi dt / h_line^2, chi dt / (dx dy)
    int n, nlines;
    int per_line, per_cross;  // periodic along the line / across lines
    int team, lines_per_block;
    int block0, nblocks;      // this job's block range in the launch
    // fixed-value (Dirichlet) boundary nodes: the first and last cell of every
    // line, and every cell of the first and last line, keep their values
    int pin_ends, pin_lines;
};

// One column update (Eq. yup) in the natural row-major layout: blocks own
// strips of `Wb` columns and all ny rows; each column is cut into `P`
// segments, one thread per (column, segment).
struct ColJob {
    const void *Tin;
    void *Tout;
    const void *TinLo;  // compensated (Kahan) low parts, or nullptr
    void *ToutLo;
    const void *g;   // cyy, face j+1/2 of column i at [j][i]
    const void *e;   // cyx
    double lam, mu;  // chi dt / dy^2, chi dt / (dx dy)
    int nx, ny;
    int per_x, per_y;
    int P, Wb;
    int block0, nblocks;
};

// Kernel arguments: either a device array of jobs (batched launches) or one
// job passed by value (jobs == nullptr).
struct LineArgs {
    const LineJob *jobs;
    int njobs;
    int limiter;
    unsigned *err;
    LineJob one;
};
struct ColArgs {
    const ColJob *jobs;
    int njobs;
    int limiter;
    unsigned *err;
    ColJob one;
};

// Vectorised contiguous-line update (line2_kernel): lines of n cells with n a
// multiple of the 16-byte vector (4 FP32 / 2 FP64 cells); output line-major
// or transposed (position-major, nlines wide).
struct Line2Job {
    const void *Tin;
    void *Tout;
    const void *TinLo;  // compensated low parts (line2, line-major output only), or nullptr
    void *ToutLo;
    const void *g;
    const void *e;
    double lam, mu;
    int n, nlines;
    int per_line, per_cross;
    int team, lines_per_block;
    int transpose_out;
    int block0, nblocks;
    // Three-dimensional lines (line4_kernel with D3): line l = kb * na + ka,
    // its neighbours along the first transverse axis are l -+ 1 (ka -+ 1),
    // along the second l -+ na (kb -+ 1); e2 and mu2 weight the limited
    // difference along the second axis.  na = 0 for two-dimensional grids.
    int na;
    const void *e2;
    double mu2;
    // Temperature-dependent diffusivity (line4_kernel with NL): the face
    // coefficients are scaled by the harmonic mean of (max(T,0) * chi_itref)^
    // chi_alpha over the two cells beside the face, T the update's input.
    double chi_alpha, chi_itref;
    // Per-step diagnostics (batched y-updates with args.diag_part set): slot
    // of this update's (sum, min, max) in the batch's ring, instance * steps + step.
    int diag_slot;
    // Compensated state on the cluster kernel (line7 with TinLo set): 1 = the
    // input (ilv_in) or output (ilv_out) is one array of quads, per line and
    // per 4 cells 4 hi values then 4 lo values (32 bytes, 2 n floats a line);
    // the TinLo / ToutLo pointers then only mark the compensated state.
    int ilv_in, ilv_out;
    // line4_kernel: shift of the shared-memory swizzle (chunk c of a line at
    // c ^ ((c >> s) & 7) within its group of 8): 0 = log2 of the chunks per
    // lane segment, 1 = none, 2..7 = s of 1..6 (line4_swizzle's choice).
    int swz;
};

// One block's diagnostics partial: FP64 sum, min and max of its lines' output.
struct DiagPart {
    double sum;
    double mn, mx;
};
struct Line2Args {
    const Line2Job *jobs;
    int njobs;
    int limiter;
    unsigned *err;
    Line2Job one;
    // optional: job index of every block of the launch (one load instead of
    // a binary search over the jobs at block start)
    const int *block_job;
    // optional (line4, 2-D): every block writes the sum, min and max of the
    // values it stores to diag_part[blockIdx.x]
    DiagPart *diag_part;
    // line4, FP32 2-D, four-warp blocks: 1 keeps each lane's gamma in tensor
    // memory (the launch's shared memory then holds two arrays, not three)
    int tmem;
};
// Finish the diagnostics of one line4 launch: for every job, the partials of
// its blocks in block order -> ring[diag_slot] = (sum, min, max).
cudaError_t launch_diag_finish(const Line2Job *jobs, int njobs, const DiagPart *part, double *ring,
                               cudaStream_t s);
// ring[0 .. count) = NaN (slots no step writes read as NaN).
cudaError_t launch_fill_nan(double *ring, size_t count, cudaStream_t s);
constexpr int MAX_LINE2_TRANSPOSED = 2048;

// Launch configuration helpers (host).
// line2: returns false when the line cannot use the vectorised kernel.
// seg_chunks: target 16-byte chunks per segment (0 = default of 4).
bool line2_config(int prec, int n, bool transposed, int *team, int *lines_per_block, int *nthreads,
                  size_t *smem, int seg_chunks = 0);
size_t line2_smem_bytes(int prec, int n, int team, int lines_per_block);
// Explicit limited step (explicit_kernel): one launch per step, blocks of
// 32 x 8 threads, each thread a column of `rows` rows.
struct ExpArgs {
    const void *Tin;
    void *Tout;
    const void *cxx, *cxy, *cyy, *cyx;
    double lamx, lamy, mu;
    int nx, ny, per;
    int rows;  // rows per thread strip
    int limiter;
    int pin;  // fixed boundary nodes (Dirichlet): the grid's outer ring keeps its values
    unsigned *err;
};
cudaError_t launch_explicit(int prec, int coef_fp16, const ExpArgs &a, cudaStream_t s);

cudaError_t launch_source(int prec, void *T, const void *Q, double dt, size_t n, cudaStream_t s);

// line4 (warp per line): returns false when the line cannot use it.
// warps: warps per block (0 = default of 4); seg_chunks: target 16-byte
// chunks per lane (0 = default of 4), which sets the team size and so the
// PCR depth.
// tmem: the tensor-memory form (FP32, four-warp blocks, at most 8 chunks a
// lane); false when the line does not fit it.
bool line4_config(int prec, int n, bool transposed, int warps, int seg_chunks, int *team, int *lines_per_block,
                  int *nthreads, size_t *smem, bool tmem = false);
cudaError_t launch_line4(int prec, int coef_fp16, const Line2Args &a, int nblocks, int nthreads,
                         size_t smem, cudaStream_t s);
// Long lines (line6): 2048 < n <= 4096, FP32, teams of 128 lanes over four
// warps, `lines` (4 or 2) lines per block.  False when the line does not fit.
bool line6_config(int prec, int coef_fp16, int n, int *team, int *lines_per_block, int *nthreads, size_t *smem,
                  int lines = 4);
cudaError_t launch_line6(int coef_fp16, const Line2Args &a, int nblocks, int nthreads, size_t smem, cudaStream_t s);
// Lines cut across a thread-block cluster (line7): FP32, n = cs * np with
// np = 2048 (else 1024) and cs = 1, 2, 4 or 8; four lines a block, one job
// (args.one) a launch; with TinLo/ToutLo set, the compensated state; with
// args.tmem (and tmem here, for the shared-memory size) each lane's gamma in
// tensor memory.  False when the line does not fit.
bool line7_config(int prec, int coef_fp16, int n, int *cs, int *nthreads, size_t *smem, bool tmem = false);
cudaError_t launch_line7(int coef_fp16, const Line2Args &a, int cs, size_t smem, cudaStream_t s);
// Resident blocks per SM of the 2-D line4 kernel for that block size and
// dynamic shared memory (CUDA's occupancy calculator; in the tensor-memory
// form also capped by the block's TMEM columns, tm_cols), or -1.
int line4_blocks_per_sm(int prec, int coef_fp16, int limiter, int nthreads, size_t smem, bool tmem = false,
                        int tm_cols = 64);
// TMEM columns a line4 block of lines of n cells (teams of `team` lanes) allocates.
int line4_tm_cols(int n, int team);
// Chunks of padding after each warp's shared area in the FP32 line4 kernel
// (narr arrays of 32/P lines of m chunks).  With teams of 16 or 8 lanes the
// two half-warps of the transposed store read lines of different warp areas;
// the pad puts those areas 16 banks apart (their offset 4 chunks mod 8).
__host__ __device__ inline int line4_area_pad(int P, int narr, int m)
{
    return P == 16 ? ((2 - 2 * narr * m) & 3) : P == 8 ? ((4 - 4 * narr * m) & 7) : 0;
}
// Line2Job::swz for a line4 line of n cells in teams of `team` lanes: the
// swizzle shift that spreads the segment phases' accesses over the shared
// memory's bank groups (fewest quarter-warp wavefronts).
int line4_swizzle(int prec, int n, int team);
// Three-dimensional grids (kernels_3d.cu).  c[0..2] = x faces (normal, with
// y, with z) in layout [nz][ny][nx]; c[3..5] = y faces (normal, with z, with
// x) in [nx][nz][ny]; c[6..8] = z faces (normal, with x, with y) in
// [ny][nx][nz].  bx, by, bz are [nz][ny][nx] in precision prec; c is in that
// precision too, or FP16 with coef_fp16 (FP32 only).
cudaError_t launch_face_coeffs3(int prec, int coef_fp16, const void *bx, const void *by, const void *bz, int nx,
                                int ny, int nz, int bc, double kappa, void *const c[9], cudaStream_t s);
// line4_kernel with the second transverse term (jobs with na > 0).
cudaError_t launch_line4_3d(int prec, int coef_fp16, const Line2Args &a, int nblocks, int nthreads, size_t smem,
                            cudaStream_t s);
void line_config(int prec, int n, int *team, int *lines_per_block, int *nthreads);
size_t line_smem_bytes(int prec, int n, int team, int lines_per_block);
void col_config(int prec, int ny, int *P, int *Wb, int *nthreads);
size_t col_smem_bytes(int prec, int ny, int P, int Wb);

// Launch wrappers (defined per precision in kernels_f32.cu / kernels_f64.cu).
// coef_fp16 selects half-precision coefficient storage (FP32 only).
// With jobs' TinLo set (FP32 only) the compensated kernels are used.
cudaError_t launch_line(int prec, int coef_fp16, const LineArgs &a, int nblocks, int nthreads,
                        size_t smem, cudaStream_t s, bool kahan = false);
cudaError_t launch_col(int prec, int coef_fp16, const ColArgs &a, int nblocks, int nthreads,
                       size_t smem, cudaStream_t s, bool kahan = false);
cudaError_t launch_line2(int prec, int coef_fp16, const Line2Args &a, int nblocks, int nthreads,
                         size_t smem, cudaStream_t s, bool kahan = false);
// Face coefficients from cell-centred b (FP64 arithmetic, one rounding to the
// storage type).  bprec: element type of bx, by.  coef: 0 fp64, 1 fp32, 2 fp16.
// cyyT/cyxT (optional) receive transposed copies [nx][ny].
cudaError_t launch_face_coeffs(int bprec, int coef, const void *bx, const void *by, int nx, int ny,
                               int bc, double kappa, void *cxx, void *cxy, void *cyy, void *cyx,
                               void *cyyT, void *cyxT, cudaStream_t s);
// out[c][r] = in[r][c] for an rows x cols array of 4- or 8-byte elements.
cudaError_t launch_transpose(int elem_bytes, const void *in, void *out, int rows, int cols,
                             cudaStream_t s);
// FP64 sum / min / max / non-finite count; partial buffers of TOTALS_BLOCKS.
constexpr int TOTALS_BLOCKS = 608;
// Tlo (optional, FP32): compensated low parts added to T in the sum.
cudaError_t launch_totals(int prec, const void *T, size_t n, double *partials, double *result,
                          cudaStream_t s, const void *Tlo = nullptr);

// Set the message aniso_last_error() returns on this host thread.
void record_error(const char *msg);

}  // namespace aniso
