// line5_kernel.cuh -- TMA-staged update of contiguous lines with the line
// state held in registers (Eq. xup on rows; Eq. yup on the column-major T*).
//
// The same delta-form line systems as line4 (the row of face p+1/2 carries
// F_p = lam g_p (T_{p+1} - T_p) + mu e_p L(v_p, v_{p+1}), v the per-cell
// inner level of the nested limiter of Eq. vanLeer), solved by the same
// segment elimination, reduced system and recovery.  What differs is where
// the data lives:
//  - one thread of the block issues five tensor-map (TMA) tile loads: the
//    block's L lines of T, the line below and the line above them, and the
//    lines' two coefficient rows.  The tiles land in shared memory in the
//    128-byte swizzled layout (16-byte chunk c of 128-byte row q at chunk
//    c ^ (q & 7)), so that the lanes of a team, each reading its own
//    contiguous segment, touch distinct bank groups;
//  - each lane then walks its segment once, top cell first: it reads the
//    three T values and two coefficients of a cell, forms the cell's inner
//    limited difference, the flux of the face above the cell and, one cell
//    behind, eliminates the row above (no flux or coefficient array is ever
//    written out).  The eliminated rows' rho stays in registers; alpha and
//    gamma overwrite the line's own coefficient tiles, which no other lane
//    reads;
//  - the segment ends are coupled by PCR over warp shuffles, as in line4;
//  - recovery forms T_new = T_old + delta in registers and stages it in the
//    g tile; after one block barrier the block writes its lines transposed
//    (position-major, `nlines` wide), L lines per store.
// The cell above a lane's segment is read directly (its inner limited
// difference is computed twice, once by each lane); the flux of the face
// below the segment comes from the lane below by one shuffle.
//
// Requirements (host side, line5_config): FP32 state and coefficients, n a
// multiple of 32 (a line is whole 128-byte rows), at most 8 chunks of 4
// cells per lane, the tensor maps of each job built over the array as rows
// of 32 floats with boxes of n/32 * L rows (T, g, e) and n/32 rows (T, one
// line).  The mbarrier wait is bounded: a block that gives up sets bit 2 of
// the error word, waits (bounded again) for its copies to land, and returns.
#pragma once
#include "line4_kernel.cuh"
#include "line5_types.h"

namespace aniso {

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of the barrier; false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// 2-D tile load (x = element in the 128-byte row, y = row) into shared memory.
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, int x, int y, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// The tensor maps live in global memory written by host copies: acquire them
// for the tensor-map proxy before use (a map at a reused address may differ
// from an earlier launch's).
__device__ __forceinline__ void tmap_acquire(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<unsigned long long>(map))
                 : "memory");
}

// Physical byte offset of logical byte offset o in a tile written with the
// 128-byte swizzle (tile base 1024-byte aligned).
__device__ __forceinline__ unsigned swz128(unsigned o) { return o ^ ((o >> 3) & 0x70u); }

// Job owning tile `tile` (jobs sorted by their first tile).
__device__ __forceinline__ int find_job5(const Line5Job *jobs, int njobs, int tile)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int line5_job_of(const Line5Args &args, int tile)
{
    return args.tile_job ? args.tile_job[tile] : find_job5(args.jobs, args.njobs, tile);
}

// Issue the five tile loads of `tile` into the stage at byte offset `st`
// (from the aligned base) on barrier `bar`.  One thread.
__device__ __forceinline__ void line5_issue(const Line5Job *Jp, int tile, unsigned base, unsigned st, unsigned bar)
{
    const int n = Jp->n, nl = Jp->nlines, L = Jp->lines_per_block;
    const int line0 = (tile - Jp->block0) * L;
    const int L_act = min(L, nl - line0);
    const Line5Smem sp = line5_smem(n, L);
    const int rows_line = n >> 5;
    const int dn = line0 > 0 ? line0 - 1 : (Jp->per_cross ? nl - 1 : 0);
    const int up = line0 + L_act < nl ? line0 + L_act : (Jp->per_cross ? 0 : nl - 1);
    const unsigned box = (unsigned)n * 4u * (unsigned)L, line = (unsigned)n * 4u;
    tmap_acquire(&Jp->tm_T);
    tmap_acquire(&Jp->tm_T1);
    tmap_acquire(&Jp->tm_g);
    tmap_acquire(&Jp->tm_e);
    mbar_expect_tx(bar, 3u * box + 2u * line);
    tma_load_2d(base + st + sp.tmain, &Jp->tm_T, 0, line0 * rows_line, bar);
    tma_load_2d(base + st + sp.g, &Jp->tm_g, 0, line0 * rows_line, bar);
    tma_load_2d(base + st + sp.e, &Jp->tm_e, 0, line0 * rows_line, bar);
    tma_load_2d(base + st + sp.tdn, &Jp->tm_T1, 0, dn * rows_line, bar);
    tma_load_2d(base + st + sp.tup, &Jp->tm_T1, 0, up * rows_line, bar);
}

__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<unsigned long long>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}
// Ask L2 for the main tiles of `tile` (T, g, e of its lines; a hint).
__device__ __forceinline__ void line5_prefetch(const Line5Job *Jp, int tile)
{
    const int row = (tile - Jp->block0) * Jp->lines_per_block * (Jp->n >> 5);
    tma_prefetch_2d(&Jp->tm_T, 0, row);
    tma_prefetch_2d(&Jp->tm_g, 0, row);
    tma_prefetch_2d(&Jp->tm_e, 0, row);
}

// UMAX: largest number of 4-cell chunks a lane owns (compile-time, so that
// the per-cell rho of the segment lives in registers).  Persistent blocks
// with two stages: while a tile is solved from one stage, the next tile of
// the block lands in the other.  The dynamic shared memory holds two stages
// of line5_smem(n_max, L).total bytes each (stage size `stage_bytes`), plus
// 1 KB for alignment.
template <int UMAX, bool VL, int STAGES = 2>
__global__ void __launch_bounds__(256, 1) line5_kernel(Line5Args args, unsigned stage_bytes)
{
    constexpr int SMAX = 4 * UMAX;
    extern __shared__ __align__(1024) unsigned char smem5_raw[];
    __shared__ __align__(8) unsigned long long s_bar[2];

    // 1024-byte aligned base inside the dynamic area (the host adds 1 KB)
    const unsigned raw = smem_addr(smem5_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    unsigned char *const sb0 = smem5_raw + (base - raw);
    const unsigned bar0 = smem_addr(&s_bar[0]), bar1 = smem_addr(&s_bar[1]);

    if (threadIdx.x == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        mbar_fence_init();
        if (!args.test_no_load && (int)blockIdx.x < args.total_tiles)
            line5_issue(args.jobs + line5_job_of(args, blockIdx.x), blockIdx.x, base, 0u, bar0);
    }
    __syncthreads();

    const int lim = args.limiter;
    const unsigned full = 0xffffffffu;
    int k = 0;  // tiles done by this block
    for (int tile = blockIdx.x; tile < args.total_tiles; tile += gridDim.x, ++k) {
    const int stage = STAGES == 2 ? (k & 1) : 0;
    const unsigned bar = stage ? bar1 : bar0;
    const unsigned phase = STAGES == 2 ? (unsigned)((k >> 1) & 1) : (unsigned)(k & 1);
    if (threadIdx.x == 0 && !args.test_no_load) {
        // with two stages the next tile of this block starts loading into the
        // other stage, freed by the barrier at the end of the previous iteration
        const int nt = tile + gridDim.x;
        if (STAGES == 2 && nt < args.total_tiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            line5_issue(args.jobs + line5_job_of(args, nt), nt, base, stage ? 0u : stage_bytes,
                        stage ? bar0 : bar1);
        }
        const int pt = tile + args.pf_dist;
        if (args.pf_dist > 0 && pt < args.total_tiles) line5_prefetch(args.jobs + line5_job_of(args, pt), pt);
    }
    unsigned char *const sb = sb0 + (stage ? stage_bytes : 0u);
    const Line5Job *Jp = args.jobs + line5_job_of(args, tile);
    const int n = Jp->n, nl = Jp->nlines, P = Jp->team, L = Jp->lines_per_block;
    const int line0 = (tile - Jp->block0) * L;
    const int L_act = min(L, nl - line0);
    const Line5Smem sp = line5_smem(n, L);
    const float lam = (float)Jp->lam, mu = (float)Jp->mu;
    const int per_line = Jp->per_line;
    const int logP = __ffs(P) - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> logP, t = lane & (P - 1);
    const int l = (warp << (5 - logP)) + q;  // line within the tile
    const bool active = l < L_act;

    // segment of lane t: chunks [c_lo, c_lo + Ut); the first rr lanes one more
    const int m = n >> 2, U = m >> logP, rr = m & (P - 1);
    const int Ut = U + (t < rr ? 1 : 0);
    const int c_lo = t * U + (t < rr ? t : rr);
    const int ct = c_lo + Ut - 1;  // top chunk
    const int e_cell = 4 * ct + 3;

    // Byte offsets from sb: tile base + logical offset of this line's row
    // (T, g and e of the line share one logical offset), and the same for the
    // lines below and above.
    const unsigned LN = (unsigned)n * 4u;
    const unsigned oc = (unsigned)l * LN;
    const unsigned tc0 = sp.tmain, tg0 = sp.g, te0 = sp.e;
    unsigned td0, od, tu0, ou;
    if (l > 0) {
        td0 = sp.tmain;
        od = oc - LN;
    } else {
        td0 = sp.tdn;
        od = 0;
    }
    if (l + 1 < L_act) {
        tu0 = sp.tmain;
        ou = oc + LN;
    } else {
        tu0 = sp.tup;
        ou = 0;
    }
    auto f4 = [sb](unsigned off) { return *reinterpret_cast<const float4 *>(sb + off); };
    auto f1 = [sb](unsigned off) { return *reinterpret_cast<const float *>(sb + off); };
    auto st4 = [sb](unsigned off, float x, float y, float z, float w) {
        *reinterpret_cast<float4 *>(sb + off) = make_float4(x, y, z, w);
    };

    // ---- wait for this tile's stage (bounded; phase k >> 1 of its barrier)
    // (the decision to give up is made for the whole block at once)
    const bool got = mbar_wait_bounded(bar, phase, args.wait_limit);
    if (__syncthreads_or(!got)) {
        if (threadIdx.x == 0) atomicOr(args.err, 2u);
        // the copies this block issued must land before it exits
        if (!args.test_no_load) {
            mbar_wait_bounded(bar, phase, 1u << 20);
            if (STAGES == 2 && tile + (int)gridDim.x < args.total_tiles)
                mbar_wait_bounded(stage ? bar0 : bar1, (unsigned)(((k + 1) >> 1) & 1), 1u << 20);
        }
        return;
    }

    // ---- the cell above the segment: T and its inner limited difference
    float Tn, vn;
    {
        int kp = e_cell + 1;
        if (kp == n) kp = per_line ? 0 : n - 1;
        const unsigned o = (unsigned)kp * 4u;
        Tn = f1(tc0 + swz128(oc + o));
        const float Tu = f1(tu0 + swz128(ou + o)), Td = f1(td0 + swz128(od + o));
        vn = level<float, VL>(lim, Tu - Tn, Tn - Td);
    }

    float rho[SMAX];  // rho[r]: row r cells below the top (r = 1 .. S-2; row S-1 is rho_s)
#pragma unroll
    for (int r = 0; r < SMAX; ++r) rho[r] = 0.f;
    float rho_s = 0.f;
    float Fn = 0.f, lgn = 0.f;                     // flux and lam*g of the face above the current cell
    float rho1 = 0.f, alp1 = 0.f, gam1 = -1.f;     // eliminated row above (row e: delta_e = X)
    float qp = 0.f, qq = 1.f, qw = 0.f;            // delta_{e-1} = qp + qq X_{t-1} + qw X_t
    float ae = 0.f, be = 1.f, ce = 0.f, re = 0.f;  // reduced row of X_t (row e)
    float Fe = 0.f, lge = 0.f;                     // face e+1/2, for the lane above
    float pa[4] = {0.f, 0.f, 0.f, 0.f}, pg[4] = {0.f, 0.f, 0.f, 0.f};  // alpha, gamma of the chunk above

    auto elim = [&](float Fk, float Fkm, float lgk, float lgkm, float &ro, float &ao, float &go) {
        // row k: -lgkm d_{k-1} + (1 + lgkm + lgk) d_k - lgk d_{k+1} = Fk - Fkm
        const float inv = Fast<float>::rcp((1.f + lgkm + lgk) + lgk * alp1);
        const float alp = -lgkm * inv, gam = lgk * gam1 * inv, rh = ((Fk - Fkm) + lgk * rho1) * inv;
        ro = rh;
        ao = alp;
        go = gam;
        qp = qp + qq * rh;
        qw = qw - qq * gam;
        qq = -qq * alp;
        rho1 = rh;
        alp1 = alp;
        gam1 = gam;
    };

    // ---- fused flux + elimination, top chunk first.  Chunk i (0 = top) is
    // chunk ct - i; its cell j (3 .. 0) is row r = 4 i + 3 - j below the top.
    // Processing row r gives the flux of the face above it and eliminates row r - 1.
#pragma unroll
    for (int i = 0; i < UMAX; ++i) {
        if (i < Ut) {
            const int c = ct - i;
            const unsigned o = (unsigned)c * 16u;
            const unsigned sc = swz128(oc + o);
            const float4 xc = f4(tc0 + sc), xd = f4(td0 + swz128(od + o)), xu = f4(tu0 + swz128(ou + o));
            const float4 xg = f4(tg0 + sc), xe = f4(te0 + sc);
            const float Tc[4] = {xc.x, xc.y, xc.z, xc.w}, Td[4] = {xd.x, xd.y, xd.z, xd.w},
                        Tu[4] = {xu.x, xu.y, xu.z, xu.w};
            const float gv[4] = {xg.x, xg.y, xg.z, xg.w}, ev[4] = {xe.x, xe.y, xe.z, xe.w};
            float na[4] = {0.f, 0.f, 0.f, 0.f}, ng[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 3; j >= 0; --j) {
                const float v = level<float, VL>(lim, Tu[j] - Tc[j], Tc[j] - Td[j]);
                const float lg = lam * gv[j];
                const float F = lg * (Tn - Tc[j]) + mu * ev[j] * level<float, VL>(lim, v, vn);
                if (i == 0 && j == 3) {  // top cell: its face flux goes to the lane above
                    Fe = F;
                    lge = lg;
                } else if (i == 0 && j == 2) {  // row e enters the reduced system
                    ae = -lg;
                    ce = -lgn;
                    be = 1.f - ae - ce;
                    re = Fn - F;
                } else {  // eliminate the row above this cell
                    float ro, ao, go;
                    elim(Fn, F, lgn, lg, ro, ao, go);
                    rho[4 * i + 2 - j] = ro;
                    if (j == 3) {  // row 0 of the chunk above: that chunk is complete
                        const unsigned sa = swz128(oc + (unsigned)(c + 1) * 16u);
                        st4(tg0 + sa, ao, pa[1], pa[2], pa[3]);
                        st4(te0 + sa, go, pg[1], pg[2], pg[3]);
                    } else {
                        na[j + 1] = ao;
                        ng[j + 1] = go;
                    }
                }
                Tn = Tc[j];
                vn = v;
                Fn = F;
                lgn = lg;
            }
            pa[1] = na[1];
            pa[2] = na[2];
            pa[3] = na[3];
            pg[1] = ng[1];
            pg[2] = ng[2];
            pg[3] = ng[3];
        }
    }

    // ---- row s (the bottom cell) needs the face below the segment: the
    // lane below's top face (the line's last face for lane 0, which wraps)
    {
        const int tp = (t - 1) & (P - 1);
        const float Fprev = __shfl_sync(full, Fe, tp, P), lgprev = __shfl_sync(full, lge, tp, P);
        float ao, go;
        elim(Fn, Fprev, lgn, lgprev, rho_s, ao, go);
        const unsigned sa = swz128(oc + (unsigned)c_lo * 16u);
        st4(tg0 + sa, ao, pa[1], pa[2], pa[3]);
        st4(te0 + sa, go, pg[1], pg[2], pg[3]);
    }

    // ---- reduced system of the line in the segment-end unknowns
    float X, Xm;
    {
        const int tn = (t + 1) & (P - 1);
        const float rho_n = __shfl_sync(full, rho1, tn, P), alp_n = __shfl_sync(full, alp1, tn, P),
                    gam_n = __shfl_sync(full, gam1, tn, P);
        X = pcr_team<float>(make_reduced<float>(ae, be, ce, re, qp, qq, qw, rho_n, alp_n, gam_n), t, P);
        Xm = __shfl_sync(full, X, (t - 1) & (P - 1), P);
    }

    // ---- recovery, bottom chunk first: delta_k = rho_k - alpha_k delta_{k-1}
    // - gamma_k X, T_new = T_old + delta, staged in the g tile
    float sum = 0.f;
    {
        float dprev = Xm;
#pragma unroll
        for (int i = UMAX - 1; i >= 0; --i) {
            if (i < Ut) {
                const int c = ct - i;
                const unsigned sc = swz128(oc + (unsigned)c * 16u);
                const float4 xa = f4(tg0 + sc), xg = f4(te0 + sc), xc = f4(tc0 + sc);
                const float a4[4] = {xa.x, xa.y, xa.z, xa.w}, g4[4] = {xg.x, xg.y, xg.z, xg.w};
                const float c4[4] = {xc.x, xc.y, xc.z, xc.w};
                float tn[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = 4 * i + 3 - j;
                    float d;
                    if (r == 0) {
                        d = X;
                    } else {
                        const float rh = (j == 0 && i == Ut - 1) ? rho_s : rho[r];
                        d = rh - a4[j] * dprev - g4[j] * X;
                    }
                    dprev = d;
                    tn[j] = c4[j] + d;
                    sum += tn[j];
                }
                st4(tg0 + sc, tn[0], tn[1], tn[2], tn[3]);
            }
        }
    }
    const bool bad = active && !(fabsf(sum) < INFINITY);

    // ---- transposed store: out[p][line0 + l], L lines per position
    __syncthreads();
    {
        float *out = static_cast<float *>(Jp->Tout);
        const bool vec = (nl & 3) == 0 && (L & 3) == 0 && L_act == L;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            float *dst = out + (size_t)p * nl + line0;
            const unsigned op = (unsigned)p * 4u;
            if (vec) {
                for (int k4 = 0; k4 < L; k4 += 4) {
                    float o4[4];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) o4[kk] = f1(tg0 + swz128((unsigned)(k4 + kk) * LN + op));
                    *reinterpret_cast<float4 *>(dst + k4) = make_float4(o4[0], o4[1], o4[2], o4[3]);
                }
            } else {
                for (int kk = 0; kk < L_act; ++kk) dst[kk] = f1(tg0 + swz128((unsigned)kk * LN + op));
            }
        }
    }
    if (bad) atomicOr(args.err, 1u);
    __syncthreads();  // the stage is free again
    if (STAGES == 1 && threadIdx.x == 0 && !args.test_no_load) {
        const int nt = tile + gridDim.x;
        if (nt < args.total_tiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            line5_issue(args.jobs + line5_job_of(args, nt), nt, base, 0u, bar0);
        }
    }
    }
}

}  // namespace aniso
