// line4_kernel.cuh -- warp-autonomous update of contiguous lines (Eq. xup on
// rows; Eq. yup on the column-major copy T*).
//
// Same linear algebra as line_sweep_kernel and line2_kernel (delta form,
// bottom-up segment elimination, PCR of the segment-end unknowns, forward
// recovery; see sweep_kernels.cuh).  What differs is the organisation:
//  - a line belongs to a team of P <= 32 lanes of one warp (32/P lines per
//    warp); no phase waits for another warp except the final transposed
//    store, so warps of a block drift apart and overlap each other's loads
//    and arithmetic;
//  - face fluxes are computed with coalesced 16-byte loads (lane t takes
//    chunks t, t+P, ..., the next round in flight during this one), the
//    limited transverse difference as Eq. vanLeer nests it: once per cell
//    v = L(T_after - T, T - T_before), then once per face L(v_p, v_{p+1}),
//    so every cell's inner value serves both of its faces;
//  - F and lam*g go to the warp's shared area, where each lane then walks
//    its own segment bottom-up (a row is eliminated as soon as the flux of
//    the face below it is known), storing (rho, alpha, gamma) in place; the
//    segment-end system is solved with warp shuffles; recovery writes delta
//    in place;
//  - T_new = T_old + delta leaves either line-major (coalesced) or,
//    staged in the same area, position-major (`nlines` wide) with the
//    lines of a block packed into 16-byte stores: the x-update writes T*
//    column-major and the y-update writes T^{n+1} back row-major.
// Shared arrays hold whole 16-byte chunks at c ^ ((c >> s) & 7) within
// complete groups of 8, so that both the chunk-parallel phases and the
// segment walks touch distinct bank groups; the host picks s per line
// (Line2Job::swz, line4_swizzle) for the segment lengths it has, the default
// being log2 of the chunks per segment.
// FP32 reciprocals use the hardware approximation (rcp.approx.ftz.f32,
// within 1 ulp); FP64 divides exactly.  Each block first asks for its input
// rows to be brought into L2 with bulk prefetches.
//
// D3: the lines of a three-dimensional grid (Section 2.1).  The face flux
// gains a second limited transverse term, mu2 * e2 * DeltaT-bar along the
// second transverse axis, from the lines -+ na away; everything after the
// flux is unchanged.  With lines along x indexed (z, y), the transposed
// output is indexed (x, z, y): the next update's lines run along y, its
// transverse axes are z then x, and its output (y, x, z) serves the
// z-update, whose output is (z, y, x) again.
#pragma once
#include "line2_kernel.cuh"

namespace aniso {

// Raw 16 bytes of T / N coefficients, converted only when used (so that a
// prefetch does not wait on its own load).
__device__ __forceinline__ float4 ld_raw(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ double2 ld_raw(const double *p) { return __ldg(reinterpret_cast<const double2 *>(p)); }
__device__ __forceinline__ uint2 ld_raw(const __half *p) { return __ldg(reinterpret_cast<const uint2 *>(p)); }
__device__ __forceinline__ void unpack_raw(const float4 &v, float *o) { V16<float>::unpack(v, o); }
__device__ __forceinline__ void unpack_raw(const double2 &v, double *o) { V16<double>::unpack(v, o); }
__device__ __forceinline__ void unpack_raw(const uint2 &v, float *o)
{
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}

// Bulk prefetch of a byte range into L2 (no destination, no completion).
__device__ __forceinline__ void l2_prefetch(const void *p, size_t bytes)
{
    if (bytes == 0 || bytes > 0xffffffffu || ((reinterpret_cast<uintptr_t>(p) | bytes) & 15)) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((unsigned)bytes) : "memory");
}

__device__ __forceinline__ float frcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <typename R> struct Fast;
template <> struct Fast<float> {
    static __device__ __forceinline__ float rcp(float x) { return frcp_approx(x); }
    static __device__ __forceinline__ float div(float a, float b) { return a * frcp_approx(b); }
};
template <> struct Fast<double> {
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
};

// One level of the nested limiter (Eq. vanLeer: L(a,b) = 2ab/(a+b) when a, b
// share a strict sign, else 0; minmod / MC as in lim2; the arithmetic mean
// for LIM_ARITH, whose nesting gives the mean of the four differences).
template <typename R> __device__ __forceinline__ R lim_level(int lim, R a, R b)
{
    if (lim == LIM_ARITH) return R(0.5) * (a + b);
    return lim2<R>(lim, a, b);
}
// van Leer in FP32: a positive product is the strict-sign test (a + b is then
// nonzero); one approximate reciprocal.
__device__ __forceinline__ float vl_level(float a, float b)
{
    const float p = a * b;
    const float r = (p + p) * frcp_approx(a + b);
    return p > 0.f ? r : 0.f;
}
template <typename R, bool VL> __device__ __forceinline__ R level(int lim, R a, R b)
{
    return lim_level<R>(lim, a, b);
}
template <> __device__ __forceinline__ float level<float, true>(int, float a, float b) { return vl_level(a, b); }

// PCR over a team of P <= 32 lanes (width-P shuffles), as pcr_warp.
template <typename R> __device__ __forceinline__ R pcr_team(Reduced<R> q, int t, int P)
{
    const unsigned full = 0xffffffffu;
    for (int h = 1; h < P; h <<= 1) {
        const int tm = (t - h) & (P - 1), tp = (t + h) & (P - 1);
        const R Lm = __shfl_sync(full, q.L, tm, P), Dm = __shfl_sync(full, q.D, tm, P);
        const R Um = __shfl_sync(full, q.U, tm, P), Rm = __shfl_sync(full, q.Rr, tm, P);
        const R Lp = __shfl_sync(full, q.L, tp, P), Dp = __shfl_sync(full, q.D, tp, P);
        const R Up = __shfl_sync(full, q.U, tp, P), Rp = __shfl_sync(full, q.Rr, tp, P);
        const R k1 = Fast<R>::div(q.L, Dm), k2 = Fast<R>::div(q.U, Dp);
        q.D = q.D - k1 * Um - k2 * Lp;
        q.Rr = q.Rr - k1 * Rm - k2 * Rp;
        q.L = -k1 * Lm;
        q.U = -k2 * Up;
    }
    return Fast<R>::div(q.Rr, q.L + q.D + q.U);
}

// Register budgets.  The FP32 2-D form asks for four resident 256-thread
// blocks' worth of registers per SM (at most 64 per thread, no spills): lines
// short enough to need little shared memory then keep up to eight 128-thread
// blocks per SM instead of five (+7 % on the uneven batch, whose launches are
// split by occupancy).  The FP32 3-D form asks for three (80 registers
// instead of 112, a few spilled values, +3 %).  FP64 keeps two: it would
// spill more than it gains.
// NL: temperature-dependent diffusivity (Section 3.3): every face's
// coefficients (normal and transverse) are scaled by the harmonic mean of
// chi(T) = (max(T,0)/t_ref)^alpha over the face's two cells, from this
// update's input T.
template <typename R> __device__ __forceinline__ R chi_pow(R x, R a);
template <> __device__ __forceinline__ float chi_pow<float>(float x, float a) { return __powf(x, a); }
template <> __device__ __forceinline__ double chi_pow<double>(double x, double a) { return pow(x, a); }
template <typename R> __device__ __forceinline__ R face_harmonic(R a, R b)
{
    return (a > R(0) && b > R(0)) ? R(2) * a * Fast<R>::div(b, a + b) : R(0);
}

// Tensor memory (TMEM) as per-thread scratch.  A block of four warps
// allocates TM_COLS columns; warp w owns TMEM lanes 32 (w % 4) .. + 31, one per
// thread, so each thread has TM_COLS private 32-bit words.  The 32x32b shape
// moves four consecutive columns of the thread's own lane per instruction
// (warp-wide, aligned).
constexpr unsigned TM_COLS = 64;
__device__ __forceinline__ void tm_alloc(unsigned *s_dst, unsigned cols = TM_COLS)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(s_dst)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(unsigned base, unsigned cols = TM_COLS)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
}
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_st4(unsigned taddr, float a, float b, float c, float d)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(__float_as_uint(a)),
                 "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d))
                 : "memory");
}
// (the load and its wait in one statement: the registers are defined on exit)
__device__ __forceinline__ void tm_ld4(unsigned taddr, float *o)
{
    unsigned r0, r1, r2, r3;
    asm volatile(
        "{\n\ttcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n\t}"
        : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
        : "r"(taddr)
        : "memory");
    o[0] = __uint_as_float(r0);
    o[1] = __uint_as_float(r1);
    o[2] = __uint_as_float(r2);
    o[3] = __uint_as_float(r3);
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// IMPL: a purely implicit update (no transverse term, mu = mu2 = 0: the second
// half-update of each axis in the 4-step scheme); neighbouring lines and
// transverse coefficients are then neither loaded nor limited.
// TM (FP32, 2-D, four-warp blocks, at most 8 chunks a lane): each lane's
// gamma lives in its TMEM lane instead of shared memory, so the line state in
// shared memory is 8 bytes a cell instead of 12 and more blocks fit an SM; the
// lane's chunks of T_old wait there too, from the flux phase to phase C
// (4 V + 4 V columns of the block's 32 or 64).
template <typename R, typename C, bool VL, bool D3 = false, bool NL = false, bool IMPL = false, bool TM = false>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? (D3 ? 3 : 4) : 2) line4_kernel(Line2Args args)
{
    static_assert(!TM || (sizeof(R) == 4 && !D3), "TMEM line state: FP32 2-D only");
    typedef typename V16<R>::T VT;
    constexpr int N = V16<R>::N;
    constexpr int LOGN = N == 4 ? 2 : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Line2Job J;
    if (args.jobs) {  // the block's job, copied by warp 0's lanes a word each
        constexpr int W8 = (int)(sizeof(Line2Job) / 8);
        static_assert(sizeof(Line2Job) % 8 == 0 && W8 <= 32, "job copy: one 8-byte word a lane");
        if (threadIdx.x < W8) {
            const int k = args.block_job ? args.block_job[blockIdx.x] : find_job(args.jobs, args.njobs);
            reinterpret_cast<unsigned long long *>(&J)[threadIdx.x] =
                reinterpret_cast<const unsigned long long *>(args.jobs + k)[threadIdx.x];
        }
    } else if (threadIdx.x == 0) {
        J = args.one;
    }
    __syncthreads();

    const int lim = args.limiter;
    const int P = J.team, n = J.n, m = n / N, nl = J.nlines, LPB = J.lines_per_block;
    const int logP = __ffs(P) - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int logL = 5 - logP;  // 32 / P lines per warp
    const int q = lane >> logP, t = lane & (P - 1);
    const int line0 = (blockIdx.x - J.block0) * LPB;
    const int line = line0 + (warp << logL) + q;
    const bool active = line < nl;
    const int lc = active ? line : nl - 1;
    int lu = lc + 1, ld = lc - 1;
    if (lu >= nl) lu = J.per_cross ? 0 : nl - 1;  // mirrored ghost line
    if (ld < 0) ld = J.per_cross ? nl - 1 : 0;
    int lbu = lc, lbd = lc;  // neighbours along the second transverse axis (D3)
    if constexpr (D3) {
        const int na = J.na, nb = nl / na, ka = lc % na, kb = lc / na;
        ld = ka > 0 ? lc - 1 : (J.per_cross ? lc + na - 1 : lc);
        lu = ka < na - 1 ? lc + 1 : (J.per_cross ? lc - (na - 1) : lc);
        lbd = kb > 0 ? lc - na : (J.per_cross ? lc + (nb - 1) * na : lc);
        lbu = kb < nb - 1 ? lc + na : (J.per_cross ? lc - (nb - 1) * na : lc);
    }
    const R *Tin = static_cast<const R *>(J.Tin);
    const R *rc = Tin + (size_t)lc * n, *ru = Tin + (size_t)lu * n, *rd = Tin + (size_t)ld * n;
    const R *rbu = Tin + (size_t)lbu * n, *rbd = Tin + (size_t)lbd * n;
    const C *G = static_cast<const C *>(J.g) + (size_t)lc * n;
    const C *E = static_cast<const C *>(J.e) + (size_t)lc * n;
    const C *E2 = D3 ? static_cast<const C *>(J.e2) + (size_t)lc * n : E;
    const R lam = (R)J.lam, mu = (R)J.mu, mu2 = (R)J.mu2;
    const R chi_a = (R)J.chi_alpha, chi_it = (R)J.chi_itref;
    auto chi_of = [chi_a, chi_it](R T_) { return T_ > R(0) ? chi_pow<R>(T_ * chi_it, chi_a) : R(0); };
    const unsigned full = 0xffffffffu;

    // The block's input rows (its lines and the two neighbouring lines of T,
    // its coefficient rows) start streaming into L2 at once, so that the
    // warps' loads below find them there.  A hint only: issued when the
    // range is 16-byte aligned.
    if (threadIdx.x == 0) {
        const int f0 = line0 > 0 && !IMPL ? line0 - 1 : line0, f1 = min(line0 + LPB + (IMPL ? 0 : 1), nl),
                  g1 = min(line0 + LPB, nl);
        l2_prefetch(Tin + (size_t)f0 * n, (size_t)(f1 - f0) * n * sizeof(R));
        l2_prefetch(static_cast<const C *>(J.g) + (size_t)line0 * n, (size_t)(g1 - line0) * n * sizeof(C));
        if constexpr (!IMPL)
            l2_prefetch(static_cast<const C *>(J.e) + (size_t)line0 * n, (size_t)(g1 - line0) * n * sizeof(C));
        if constexpr (D3 && !IMPL) {
            l2_prefetch(static_cast<const C *>(J.e2) + (size_t)line0 * n, (size_t)(g1 - line0) * n * sizeof(C));
            // the block's neighbours along the second transverse axis, where not wrapped
            if (line0 >= J.na) l2_prefetch(Tin + (size_t)(line0 - J.na) * n, (size_t)(g1 - line0) * n * sizeof(R));
            if (g1 + J.na <= nl) l2_prefetch(Tin + (size_t)(line0 + J.na) * n, (size_t)(g1 - line0) * n * sizeof(R));
        }
    }

    // segment of lane t: chunks [c_lo, c_lo + Ut); the first rr lanes one more
    const int U = m >> logP, rr = m & (P - 1);
    const int Ut = U + (t < rr ? 1 : 0);
    const int c_lo = t * U + (t < rr ? t : rr);
    const int V = U + (rr ? 1 : 0);  // chunk rounds of the coalesced phases
    const int WA = m << logL;        // chunks per array in one warp's area
    const int mfull = m & ~7, logU = 31 - __clz(U);
    constexpr int NARR = TM ? 2 : 3;  // shared arrays per warp area
    const int AS = NARR * WA + (N == 4 ? line4_area_pad(P, NARR, m) : 0);  // chunks per warp area
    VT *wbase = reinterpret_cast<VT *>(smem_raw) + (size_t)warp * AS;
    VT *sA = wbase + q * m;           // F -> rho -> delta -> T_new
    VT *sB = wbase + WA + q * m;      // lam*g -> alpha
    VT *sC = wbase + 2 * WA + q * m;  // gamma (shared-memory form only)
    // TMEM form: the block's columns (32 when a lane's 4 V + 4 fit, so that
    // more blocks share an SM's 512), this warp's lane quarter
    // (warp 0 allocates now; the address is read after the barrier that
    // follows the first round's loads, so the allocation overlaps them)
    __shared__ unsigned s_tmem;
    unsigned tm_base = 0, tm_lane = 0;
    const unsigned tm_cols = 8 * V <= 32 ? 32u : 64u;
    if constexpr (TM) {
        if (warp == 0) tm_alloc(&s_tmem, tm_cols);
        tm_fence_before();
    }
    const int swsh = J.swz >= 2 ? J.swz - 1 : logU;
    const int swmk = J.swz == 1 ? 0 : 7;
    auto swz = [mfull, swsh, swmk](int c) { return c < mfull ? c ^ ((c >> swsh) & swmk) : c; };

    // ---- A: face fluxes and lam*g, coalesced (lane t: chunks v*P + t), last round first
    {
        const VT *vd = reinterpret_cast<const VT *>(rd), *vc = reinterpret_cast<const VT *>(rc),
                 *vu = reinterpret_cast<const VT *>(ru);
        const VT *vbd = reinterpret_cast<const VT *>(rbd), *vbu = reinterpret_cast<const VT *>(rbu);
        R Tcar = R(0), vcar = R(0);  // cell 0 of chunk (v+1)P, from the team's lane 0
        R wcar = R(0);               // the same for the second transverse axis (D3)
        // the next round's loads are issued before this round's arithmetic
        int cl = min(((V - 1) << logP) + t, m - 1);
        VT xc = vc[cl], xd = xc, xu = xc;
        auto xg = ld_raw(G + cl * N), xe = xg;
        if constexpr (!IMPL) {
            xd = vd[cl];
            xu = vu[cl];
            xe = ld_raw(E + cl * N);
        }
        VT xbd = xc, xbu = xc;
        auto xe2 = xe;
        if constexpr (D3 && !IMPL) {
            xbd = vbd[cl];
            xbu = vbu[cl];
            xe2 = ld_raw(E2 + cl * N);
        }
        // the cell after the line (periodic wrap or mirrored ghost), issued
        // with the first round's loads instead of inside that round (2-D; the
        // 3-D and temperature-dependent forms, short of registers, load it
        // where it is used)
        constexpr bool EARLY = !D3 && !NL;
        const int p1 = J.per_line ? 0 : n - 1;
        R eT = R(0), eU = R(0), eD = R(0);
        if constexpr (EARLY) {
            eT = rc[p1];
            if constexpr (!IMPL) {
                eU = ru[p1];
                eD = rd[p1];
            }
        }
        if constexpr (TM) {  // the block's TMEM address, the first loads in flight
            __syncthreads();
            tm_fence_after();
            tm_base = s_tmem;
            tm_lane = tm_base + ((unsigned)(32 * (warp & 3)) << 16);
        }
        for (int v = V - 1; v >= 0; --v) {
            const int c = (v << logP) + t;
            R Td[N], Tc[N], Tu[N], Gv[N], Ev[N], Tbd[N], Tbu[N], E2v[N];
            V16<R>::unpack(xc, Tc);
            // TMEM form: this chunk of T_old waits in the lane's columns 4 (V + v)
            // for phase C, which takes the same chunks by the same lanes
            if constexpr (TM) tm_st4(tm_lane + 4u * (unsigned)(V + v), Tc[0], Tc[1], Tc[2], Tc[3]);
            unpack_raw(xg, Gv);
            if constexpr (!IMPL) {
                V16<R>::unpack(xd, Td);
                V16<R>::unpack(xu, Tu);
                unpack_raw(xe, Ev);
            }
            if constexpr (D3 && !IMPL) {
                V16<R>::unpack(xbd, Tbd);
                V16<R>::unpack(xbu, Tbu);
                unpack_raw(xe2, E2v);
            }
            const int cur = cl;
            if (v > 0) {
                cl = ((v - 1) << logP) + t;  // always < m
                xc = vc[cl];
                xg = ld_raw(G + cl * N);
                if constexpr (!IMPL) {
                    xd = vd[cl];
                    xu = vu[cl];
                    xe = ld_raw(E + cl * N);
                }
                if constexpr (D3 && !IMPL) {
                    xbd = vbd[cl];
                    xbu = vbu[cl];
                    xe2 = ld_raw(E2 + cl * N);
                }
            }
            R vv[N], ww[N];
            if constexpr (!IMPL) {
#pragma unroll
                for (int j = 0; j < N; ++j) vv[j] = level<R, VL>(lim, Tu[j] - Tc[j], Tc[j] - Td[j]);
            }
            if constexpr (D3 && !IMPL) {
#pragma unroll
                for (int j = 0; j < N; ++j) ww[j] = level<R, VL>(lim, Tbu[j] - Tc[j], Tc[j] - Tbd[j]);
            }
            R nT = __shfl_down_sync(full, Tc[0], 1, P), nv = R(0), nw = R(0);
            if constexpr (!IMPL) nv = __shfl_down_sync(full, vv[0], 1, P);
            if constexpr (D3 && !IMPL) nw = __shfl_down_sync(full, ww[0], 1, P);
            if (t == P - 1) {
                nT = Tcar;
                nv = vcar;
                nw = wcar;
            }
            if (cur == m - 1) {  // the cell after the line
                if constexpr (!EARLY) {
                    nT = rc[p1];
                    if constexpr (!IMPL) nv = level<R, VL>(lim, ru[p1] - nT, nT - rd[p1]);
                    if constexpr (D3 && !IMPL) nw = level<R, VL>(lim, rbu[p1] - nT, nT - rbd[p1]);
                } else {
                    nT = eT;
                    if constexpr (!IMPL) nv = level<R, VL>(lim, eU - nT, nT - eD);
                }
            }
            Tcar = __shfl_sync(full, Tc[0], 0, P);
            if constexpr (!IMPL) vcar = __shfl_sync(full, vv[0], 0, P);
            if constexpr (D3 && !IMPL) wcar = __shfl_sync(full, ww[0], 0, P);
            R F[N], lg[N], hf[N];
            if constexpr (NL) {
                R ch[N + 1];
#pragma unroll
                for (int j = 0; j < N; ++j) ch[j] = chi_of(Tc[j]);
                ch[N] = chi_of(nT);
#pragma unroll
                for (int j = 0; j < N; ++j) hf[j] = face_harmonic<R>(ch[j], ch[j + 1]);
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const R Tnx = j + 1 < N ? Tc[j + 1] : nT;
                const R gj = NL ? Gv[j] * hf[j] : Gv[j];
                lg[j] = lam * gj;
                if constexpr (IMPL) {
                    F[j] = lg[j] * (Tnx - Tc[j]);
                } else {
                    const R vnx = j + 1 < N ? vv[j + 1] : nv;
                    const R ej = NL ? Ev[j] * hf[j] : Ev[j];
                    F[j] = lg[j] * (Tnx - Tc[j]) + mu * ej * level<R, VL>(lim, vv[j], vnx);
                }
                if constexpr (D3 && !IMPL) {
                    const R wnx = j + 1 < N ? ww[j + 1] : nw;
                    F[j] += mu2 * (NL ? E2v[j] * hf[j] : E2v[j]) * level<R, VL>(lim, ww[j], wnx);
                }
            }
            if (c < m) {
                sA[swz(c)] = V16<R>::pack(F);
                sB[swz(c)] = V16<R>::pack(lg);
            }
        }
    }
    __syncwarp();

    // ---- B1: bottom-up elimination of lane t's segment
    R rho1 = R(0), alp1 = R(0), gam1 = R(-1);
    R qp = R(0), qq = R(1), qw = R(0);
    R ae = R(0), be = R(1), ce = R(0), re = R(0);
    {
        auto elim = [&](R Fk, R Fkm, R lgk, R lgkm, R &ro_, R &ao_, R &go_) {
            // row k: -lgkm d_{k-1} + (1 + lgkm + lgk) d_k - lgk d_{k+1} = Fk - Fkm
            const R inv = Fast<R>::rcp((R(1) + lgkm + lgk) + lgk * alp1);
            const R alp = -lgkm * inv, gam = lgk * gam1 * inv, rho = ((Fk - Fkm) + lgk * rho1) * inv;
            ro_ = rho;
            ao_ = alp;
            go_ = gam;
            qp = qp + qq * rho;
            qw = qw - qq * gam;
            qq = -qq * alp;
            rho1 = rho;
            alp1 = alp;
            gam1 = gam;
        };
        R Fpend = R(0), lgpend = R(0), Flast = R(0), lglast = R(0);
        R ro[N], ao[N], go[N];  // maps of the chunk above, waiting for its row 0
#pragma unroll
        for (int v = 0; v < N; ++v) ro[v] = ao[v] = go[v] = R(0);
        // (TMEM form: every lane runs all V rounds, so that the warp-wide TMEM
        // stores stay uniform; a lane's rounds past its segment do nothing but
        // store to columns its segment does not use)
        for (int u = TM ? V - 1 : Ut - 1; u >= 0; --u) {
            R gs[N];  // gamma of the chunk above once its row 0 is eliminated (TMEM form)
#pragma unroll
            for (int j = 0; j < N; ++j) gs[j] = R(0);
            if (!TM || u < Ut) {
            const int c = c_lo + u;
            R F[N], lg[N], co[N], cao[N], cgo[N];
            V16<R>::unpack(sA[swz(c)], F);
            V16<R>::unpack(sB[swz(c)], lg);
            if (u == Ut - 1) {
                // row e (last cell of the segment) enters the reduced system
                ae = -lg[N - 2];
                ce = -lg[N - 1];
                be = R(1) - ae - ce;
                re = F[N - 1] - F[N - 2];
                Flast = F[N - 1];
                lglast = lg[N - 1];
                co[N - 1] = cao[N - 1] = cgo[N - 1] = R(0);
#pragma unroll
                for (int j = N - 2; j >= 1; --j) elim(F[j], F[j - 1], lg[j], lg[j - 1], co[j], cao[j], cgo[j]);
            } else {
                // row 0 of the chunk above, then this chunk's rows N-1 .. 1
                elim(Fpend, F[N - 1], lgpend, lg[N - 1], ro[0], ao[0], go[0]);
                sA[swz(c + 1)] = V16<R>::pack(ro);
                sB[swz(c + 1)] = V16<R>::pack(ao);
                if constexpr (TM) {
#pragma unroll
                    for (int j = 0; j < N; ++j) gs[j] = go[j];
                } else {
                    sC[swz(c + 1)] = V16<R>::pack(go);
                }
#pragma unroll
                for (int j = N - 1; j >= 1; --j) elim(F[j], F[j - 1], lg[j], lg[j - 1], co[j], cao[j], cgo[j]);
            }
            Fpend = F[0];
            lgpend = lg[0];
#pragma unroll
            for (int j = 1; j < N; ++j) {
                ro[j] = co[j];
                ao[j] = cao[j];
                go[j] = cgo[j];
            }
            }
            // (chunk u + 1's gamma at columns 4 (u + 1); in the first round there is none)
            if constexpr (TM)
                if (u + 1 < V) tm_st4(tm_lane + 4u * (unsigned)(u + 1), gs[0], gs[1], gs[2], gs[3]);
        }
        // row s needs the face below the segment: the previous lane's last face
        const int tp = (t - 1) & (P - 1);
        const R Fprev = __shfl_sync(full, Flast, tp, P), lgprev = __shfl_sync(full, lglast, tp, P);
        elim(Fpend, Fprev, lgpend, lgprev, ro[0], ao[0], go[0]);
        sA[swz(c_lo)] = V16<R>::pack(ro);
        sB[swz(c_lo)] = V16<R>::pack(ao);
        if constexpr (TM) {
            tm_st4(tm_lane, go[0], go[1], go[2], go[3]);
            tm_wait_st();  // the recovery below reads these columns back
        } else {
            sC[swz(c_lo)] = V16<R>::pack(go);
        }
    }

    // Phase C's first two chunks of T_old start loading now, so that their
    // latency hides behind R and B2 (-3 to -4 % measured on 1024-cell lines).
    // (TMEM form: T_old is in tensor memory already)
    const VT *vcC = reinterpret_cast<const VT *>(rc);
    VT pre0{}, pre1{};
    if constexpr (!TM) {
        pre0 = pre1 = vcC[t];  // t < P <= m
        if (t + P < m) pre1 = vcC[t + P];
    }

    // ---- R: reduced system of the line in the segment-end unknowns
    R X, Xm;
    {
        const int tn = (t + 1) & (P - 1);
        const R rho_n = __shfl_sync(full, rho1, tn, P), alp_n = __shfl_sync(full, alp1, tn, P),
                gam_n = __shfl_sync(full, gam1, tn, P);
        X = pcr_team<R>(make_reduced<R>(ae, be, ce, re, qp, qq, qw, rho_n, alp_n, gam_n), t, P);
        Xm = __shfl_sync(full, X, (t - 1) & (P - 1), P);
    }

    // ---- B2: forward recovery of lane t's segment (delta over rho)
    {
        R dprev = Xm;
        for (int u = 0; u < (TM ? V : Ut); ++u) {
            R g4[N];
            if constexpr (TM) tm_ld4(tm_lane + 4u * (unsigned)u, reinterpret_cast<float *>(g4));  // warp-wide
            if (TM && u >= Ut) continue;
            const int c = c_lo + u;
            R r4[N], a4[N], d[N];
            V16<R>::unpack(sA[swz(c)], r4);
            V16<R>::unpack(sB[swz(c)], a4);
            if constexpr (!TM) V16<R>::unpack(sC[swz(c)], g4);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                d[j] = (u == Ut - 1 && j == N - 1) ? X : r4[j] - a4[j] * dprev - g4[j] * X;
                dprev = d[j];
            }
            sA[swz(c)] = V16<R>::pack(d);
        }
    }
    __syncwarp();

    // ---- C: T_new = T_old + delta, coalesced
    bool bad = false;
    // diagnostics: compensated sum of the chunk sums, min, max of this lane's cells
    const bool diag = args.diag_part != nullptr;
    R dh = R(0), dl = R(0), dmn = R(INFINITY), dmx = R(-INFINITY);
    {
        VT *vout = reinterpret_cast<VT *>(static_cast<R *>(J.Tout) + (size_t)lc * n);
        for (int v = 0; v < V; ++v) {
            const int c = (v << logP) + t;
            R to[N], d[N];
            if constexpr (TM) {
                tm_ld4(tm_lane + 4u * (unsigned)(V + v), to);  // warp-wide, before the lane's bound check
                if (c >= m) continue;
            } else {
                if (c >= m) break;
                V16<R>::unpack(pre0, to);
                pre0 = pre1;  // two chunks in flight
                if (c + 2 * P < m) pre1 = vcC[c + 2 * P];
            }
            V16<R>::unpack(sA[swz(c)], d);
            R sum = R(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                to[j] += d[j];
                sum += to[j];
            }
            bad |= !(fabs(sum) < R(INFINITY));  // a NaN or infinity in the chunk
            if (diag && active) {
                const R y = sum - dl, tt = dh + y;
                dl = (tt - dh) - y;
                dh = tt;
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    dmn = fmin(dmn, to[j]);
                    dmx = fmax(dmx, to[j]);
                }
            }
            if (!J.transpose_out) {
                if (active) vout[c] = V16<R>::pack(to);
            } else {
                sA[swz(c)] = V16<R>::pack(to);
            }
        }
    }

    // ---- transposed store: out[p][line], N lines per 16-byte store.  With
    // two or more line groups a block (short lines), lanes l and l + 16 of a
    // warp write neighbouring groups of one position, so that each store
    // instruction fills whole 32-byte sectors (16 positions x 2 groups).
    if (J.transpose_out) {
        __syncthreads();
        R *out = static_cast<R *>(J.Tout);
        const int groups = LPB >> LOGN, logG = __ffs(groups) - 1;
        const bool vec_ok = (nl & (N - 1)) == 0;
        const int pairs = groups == 1 ? n : (((n + 15) & ~15) << logG);
        for (int idx = threadIdx.x; idx < pairs; idx += blockDim.x) {
            const int p = groups == 1 ? idx : (((idx >> (4 + logG)) << 4) | (idx & 15));
            const int grp = groups == 1 ? 0 : ((idx >> 4) & (groups - 1));
            if (p >= n) continue;
            const int sc = swz(p >> LOGN), j = p & (N - 1);
            {
                R o[N];
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const int lb = (grp << LOGN) + i;
                    const VT *src = reinterpret_cast<const VT *>(smem_raw) + (size_t)(lb >> logL) * AS +
                                    (lb & ((1 << logL) - 1)) * m + sc;
                    o[i] = reinterpret_cast<const R *>(src)[j];
                }
                const int l0 = line0 + (grp << LOGN);
                R *dst = out + (size_t)p * nl + l0;
                if (vec_ok && l0 + N <= nl) {
                    *reinterpret_cast<VT *>(dst) = V16<R>::pack(o);
                } else {
#pragma unroll
                    for (int i = 0; i < N; ++i)
                        if (l0 + i < nl) dst[i] = o[i];
                }
            }
        }
    }
    if (bad && active) atomicOr(args.err, 1u);
    if (diag) {  // the block's partial, reduced in a fixed order (deterministic)
        __shared__ DiagPart s_diag[8];
        double ds = (double)dh - (double)dl, mn = (double)dmn, mx = (double)dmx;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ds += __shfl_xor_sync(full, ds, o);
            mn = fmin(mn, __shfl_xor_sync(full, mn, o));
            mx = fmax(mx, __shfl_xor_sync(full, mx, o));
        }
        if (lane == 0) s_diag[warp] = DiagPart{ds, mn, mx};
        __syncthreads();
        if (threadIdx.x == 0) {
            DiagPart p = s_diag[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                p.sum += s_diag[w].sum;
                p.mn = fmin(p.mn, s_diag[w].mn);
                p.mx = fmax(p.mx, s_diag[w].mx);
            }
            args.diag_part[blockIdx.x] = p;
        }
    }
    if constexpr (TM) {  // every warp is done with TMEM before the block frees it
        tm_fence_before();
        __syncthreads();
        if (warp == 0) {
            tm_fence_after();
            tm_dealloc(tm_base, tm_cols);
        }
    }
}

}  // namespace aniso
