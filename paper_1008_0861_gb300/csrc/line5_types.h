// line5_types.h -- job, argument and shared-memory plan of the TMA-staged
// line kernel (line5_kernel.cuh), shared with the host code that builds the
// batched plans.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace aniso {

struct alignas(128) Line5Job {
    CUtensorMap tm_T;   // T lines, box {32, n/32 * L}
    CUtensorMap tm_T1;  // T lines, box {32, n/32}: one line
    CUtensorMap tm_g;   // normal coefficient, box {32, n/32 * L}
    CUtensorMap tm_e;   // transverse coefficient, same box
    void *Tout;         // transposed output, [n][nlines]
    double lam, mu;
    int n, nlines;
    int per_line, per_cross;
    int team, lines_per_block;
    int block0, nblocks;
};

// A launch covers the tiles (groups of `lines_per_block` lines) of all its
// jobs, numbered from 0 to total_tiles - 1 (job tiles start at block0);
// each block walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
struct Line5Args {
    const Line5Job *jobs;  // device array sorted by block0 (128-byte aligned)
    int njobs;
    int total_tiles;
    int limiter;
    unsigned *err;
    unsigned wait_limit;  // tries of the bounded wait for a tile
    int test_no_load;     // 1: issue no loads, so that the first wait gives up (failure-path test)
    int pf_dist;          // > 0: each tile also asks L2 for the tiles of tile + pf_dist (a hint)
    const int *tile_job;  // optional: job index of every tile (else a binary search)
};

// Shared-memory plan of a block (bytes from a 1024-byte aligned base).
struct Line5Smem {
    unsigned tmain, tdn, tup, g, e, total;
};
__host__ __device__ inline unsigned round1k(unsigned v) { return (v + 1023u) & ~1023u; }
__host__ __device__ inline Line5Smem line5_smem(int n, int L)
{
    Line5Smem s;
    const unsigned line = (unsigned)n * 4u, box = line * (unsigned)L;
    s.tmain = 0;
    s.tdn = round1k(box);
    s.tup = s.tdn + round1k(line);
    s.g = s.tup + round1k(line);
    s.e = s.g + round1k(box);
    s.total = s.e + round1k(box);
    return s;
}

// Host side (kernels_line5.cu).
// True when the driver offers tensor-map encoding.
bool line5_available();
// Block shape of a line of n cells: false when line5 cannot take it.
bool line5_config(int prec, int coef_fp16, int n, int *team, int *lines_per_block, int *nthreads, size_t *stage);
// Tensor maps of job J (n, lines_per_block set): T lines, g, e arrays of `cells` floats.
bool line5_make_maps(Line5Job &J, const void *Tin, const void *g, const void *e, size_t cells);
// Before any stream capture: set the kernel's shared-memory limit for a
// launch of that shape and return its resident blocks on the device (-1 on
// error); the batch uses it as the L2 prefetch distance (a.pf_dist).
int line5_prepare(int limiter, int nthreads, size_t stage);
// One launch over all tiles of a.jobs; stage: the largest job's line5_smem().total.
cudaError_t launch_line5(const Line5Args &a, int nthreads, size_t stage, cudaStream_t s);

}  // namespace aniso
