// line3_kernel.cuh -- persistent, bulk-copy-staged contiguous-line update
// (Eq. xup on rows; Eq. yup on the column-major copy of T*).
//
// Arithmetic and shared-memory working layout are those of line2_kernel
// (delta form, segment elimination, PCR of the segment-end unknowns, chunk
// swizzle).  What changes is how the inputs arrive:
//  - blocks are persistent and walk "groups" of LPB consecutive lines;
//  - the rows a group needs (T of lines line0-1 .. line0+LPB, and the two
//    coefficient rows of each line) are fetched by one thread with 1-D bulk
//    asynchronous copies (cp.async.bulk ... mbarrier::complete_tx) into a
//    dense staging area, completion signalled on an mbarrier;
//  - as soon as phase A has turned the staged rows into fluxes, the copies of
//    the block's next group are issued, so HBM traffic for group k+1 overlaps
//    the solve and the output of group k.
// Every mbarrier wait is bounded; on timeout the block raises bit 2 of the
// error word, waits (bounded) for its own copies still in flight and returns.
#pragma once
#include "line2_kernel.cuh"

namespace aniso {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: at most 2^22 polls (each may suspend the thread briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

constexpr unsigned ERR_TIMEOUT_BIT = 2u;

// Shared-memory plan of one group (host computes the same numbers).
struct Line3Plan {
    int stageT, stageG, stageE;  // byte offsets of the staging arrays
    int work;                    // byte offset of the working arrays
    int bytes;                   // total dynamic shared memory
};

template <typename R, typename C>
__host__ __device__ inline Line3Plan line3_plan(int n, int team, int lpb)
{
    constexpr int N = 16 / sizeof(R);
    Line3Plan p;
    const int rowT = n * (int)sizeof(R), rowC = n * (int)sizeof(C);
    auto up16 = [](int b) { return (b + 15) & ~15; };
    p.stageT = 0;
    p.stageG = up16(p.stageT + (lpb + 2) * rowT);
    p.stageE = up16(p.stageG + lpb * rowC);
    p.work = up16(p.stageE + lpb * rowC);
    int work_words = lpb * (3 * n + N) + (team > 32 ? lpb * 8 * team : 0);
    p.bytes = p.work + work_words * (int)sizeof(R);
    return p;
}

template <typename R, typename C>
__global__ void __launch_bounds__(512, 2) line3_kernel(Line3Args args)
{
    typedef typename V16<R>::T VT;
    constexpr int N = V16<R>::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Line3Job Jbuf[2];
    __shared__ __align__(8) uint64_t bar;
    const unsigned full = 0xffffffffu;
    const int total = args.total_groups;

    // map a line index (possibly a ghost) of job J to a stored line
    // (a group may extend past the last line when the grid has fewer lines
    // than a block holds, so wrap with a true modulo and clamp otherwise)
    auto map_line = [](const Line3Job &J, int x) {
        if (x >= 0 && x < J.nlines) return x;
        if (J.per_cross) return ((x % J.nlines) + J.nlines) % J.nlines;
        return x < 0 ? 0 : J.nlines - 1;
    };
    auto job_for = [&](int gidx) -> Line3Job {
        if (!args.jobs) return args.one;
        int lo = 0, hi = args.njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (args.jobs[mid].group0 <= gidx) lo = mid;
            else hi = mid - 1;
        }
        return args.jobs[lo];
    };
    // thread 0: stage the rows of group gidx (job J) into the staging area
    auto issue = [&](const Line3Job &J, int gidx) {
        const Line3Plan pl = line3_plan<R, C>(J.n, J.team, J.lines_per_block);
        const int LPB = J.lines_per_block, n = J.n;
        const int line0 = (gidx - J.group0) * LPB;
        const uint32_t rowT = n * sizeof(R), rowC = n * sizeof(C);
        fence_proxy_async_smem();  // earlier generic accesses to the staging area before the async writes
        mbar_arrive_expect_tx(&bar, (LPB + 2) * rowT + 2 * LPB * rowC);
        const R *Tin = static_cast<const R *>(J.Tin);
        for (int r = 0; r < LPB + 2; ++r) {
            const int ln = map_line(J, line0 - 1 + r);
            bulk_g2s(smem_raw + pl.stageT + r * rowT, Tin + (size_t)ln * n, rowT, &bar);
        }
        const C *G = static_cast<const C *>(J.g), *E = static_cast<const C *>(J.e);
        for (int r = 0; r < LPB; ++r) {
            const int ln = line0 + r < J.nlines ? line0 + r : J.nlines - 1;
            bulk_g2s(smem_raw + pl.stageG + r * rowC, G + (size_t)ln * n, rowC, &bar);
            bulk_g2s(smem_raw + pl.stageE + r * rowC, E + (size_t)ln * n, rowC, &bar);
        }
    };

    int gidx = blockIdx.x;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (gidx < total) {
            Jbuf[0] = job_for(gidx);
            issue(Jbuf[0], gidx);
        }
    }
    __syncthreads();
    uint32_t parity = 0;
    int cur = 0;
    bool bad = false;

    for (; gidx < total; gidx += gridDim.x) {
        const Line3Job &J = Jbuf[cur];
        // ---- wait for this group's rows
        const bool ok = mbar_wait_bounded(&bar, parity);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(args.err, ERR_TIMEOUT_BIT);
                mbar_wait_bounded(&bar, parity);  // let copies still in flight land
            }
            __syncthreads();
            return;
        }
        parity ^= 1u;

        const int lim = args.limiter;
        const int P = J.team, n = J.n, m = n / N, nl = J.nlines, LPB = J.lines_per_block;
        const int logP = __ffs(P) - 1;
        const int tm = threadIdx.x >> logP, t = threadIdx.x & (P - 1);
        const int line0 = (gidx - J.group0) * LPB;
        const int line = line0 + tm;
        const bool active = line < nl;
        const int lc = active ? line : nl - 1;
        const Line3Plan pl = line3_plan<R, C>(n, P, LPB);
        const int work_off = args.work_off;  // common to all jobs of the launch
        const R lam = (R)J.lam, mu = (R)J.mu;
        const bool per_line = J.per_line != 0;
        const R *Tin = static_cast<const R *>(J.Tin);
        const R *rd = reinterpret_cast<const R *>(smem_raw + pl.stageT) + (size_t)tm * n;  // staged line-1
        const R *rc = rd + n, *ru = rd + 2 * n;
        const C *G = reinterpret_cast<const C *>(smem_raw + pl.stageG) + (size_t)tm * n;
        const C *E = reinterpret_cast<const C *>(smem_raw + pl.stageE) + (size_t)tm * n;

        const int LS = 3 * n + N;
        R *sF = reinterpret_cast<R *>(smem_raw + work_off) + tm * LS;
        R *sG = sF + n;
        R *sQ = sG + n;
        VT *vF = reinterpret_cast<VT *>(sF), *vG = reinterpret_cast<VT *>(sG), *vQ = reinterpret_cast<VT *>(sQ);
        const int mfull = m & ~7;
        auto swz = [mfull](int c) { return swz_chunk(c, mfull); };
        auto at = [&](int k) { return swz(k / N) * N + (k & (N - 1)); };

        // ---- A: staged rows -> face fluxes and normal coefficients (swizzled)
        {
            const int width = P < 32 ? P : 32;
            const int lane_in = t & (width - 1);
            const VT *vd = reinterpret_cast<const VT *>(rd), *vc = reinterpret_cast<const VT *>(rc),
                     *vu = reinterpret_cast<const VT *>(ru);
            for (int c0 = 0; c0 < m; c0 += P) {
                const int c = c0 + t;
                const int cl = c < m ? c : m - 1;
                R Td[N], Tc[N], Tu[N], Gv[N], Ev[N];
                V16<R>::unpack(vd[cl], Td);
                V16<R>::unpack(vc[cl], Tc);
                V16<R>::unpack(vu[cl], Tu);
                ld_coef_chunk_smem(G + cl * N, Gv);
                ld_coef_chunk_smem(E + cl * N, Ev);
                R nd = __shfl_down_sync(full, Td[0], 1, width);
                R nc = __shfl_down_sync(full, Tc[0], 1, width);
                R nu = __shfl_down_sync(full, Tu[0], 1, width);
                if (c < m) {
                    if (lane_in == width - 1 || c + 1 >= m) {
                        int p1 = (c + 1) * N;
                        if (p1 >= n) p1 = per_line ? 0 : n - 1;
                        nd = rd[p1];
                        nc = rc[p1];
                        nu = ru[p1];
                    }
                    R Fo[N];
#pragma unroll
                    for (int v = 0; v < N; ++v) {
                        const R d1 = v + 1 < N ? Td[v + 1] : nd;
                        const R c1 = v + 1 < N ? Tc[v + 1] : nc;
                        const R u1 = v + 1 < N ? Tu[v + 1] : nu;
                        const R dT = limit4_v2<R>(lim, u1 - c1, c1 - d1, Tu[v] - Tc[v], Tc[v] - Td[v]);
                        Fo[v] = lam * Gv[v] * (c1 - Tc[v]) + mu * Ev[v] * dT;
                    }
                    vF[swz(c)] = V16<R>::pack(Fo);
                    vG[swz(c)] = V16<R>::pack(Gv);
                }
            }
        }
        __syncthreads();

        // ---- staging area free: fetch the next group's rows while this one is solved
        const int gnext = gidx + gridDim.x;
        if (threadIdx.x == 0 && gnext < total) {
            Jbuf[cur ^ 1] = job_for(gnext);
            issue(Jbuf[cur ^ 1], gnext);
        }

        // ---- B1 / R / B2 (as line2_kernel)
        const int c_lo = (t * m) >> logP, c_hi = ((t + 1) * m) >> logP;
        const int s = c_lo * N;
        {
            const int sm1 = s == 0 ? n - 1 : s - 1;
            const R Fsm1 = sF[at(sm1)], gsm1 = sG[at(sm1)];
            if (P > 32) __syncthreads();
            else __syncwarp();
            R rho1 = R(0), alp1 = R(0), gam1 = R(-1);
            R qp = R(0), qq = R(1), qw = R(0);
            R ae, be, ce, re;
            R f[N] = {}, gg[N] = {}, fp[N] = {}, gp[N] = {};
            auto load_prev = [&](int cc) {
                if (cc > c_lo) {
                    V16<R>::unpack(vF[swz(cc - 1)], fp);
                    V16<R>::unpack(vG[swz(cc - 1)], gp);
                } else {
                    fp[N - 1] = Fsm1;
                    gp[N - 1] = gsm1;
                }
            };
            auto eliminate = [&](int v, R Fkm, R gkm, R *ro, R *ao, R *go) {
                const R a = -lam * gkm, c = -lam * gg[v];
                const R b = R(1) - a - c;
                const R inv = Num<R>::div(R(1), b - c * alp1);
                const R alp = a * inv, gam = -c * gam1 * inv, rho = (f[v] - Fkm - c * rho1) * inv;
                ro[v] = rho;
                ao[v] = alp;
                go[v] = gam;
                qp = qp + qq * rho;
                qw = qw - qq * gam;
                qq = -qq * alp;
                rho1 = rho;
                alp1 = alp;
                gam1 = gam;
            };
            int cc = c_hi - 1;
            V16<R>::unpack(vF[swz(cc)], f);
            V16<R>::unpack(vG[swz(cc)], gg);
            load_prev(cc);
            {
                R ro[N], ao[N], go[N];
                ae = -lam * gg[N - 2];
                ce = -lam * gg[N - 1];
                be = R(1) - ae - ce;
                re = f[N - 1] - f[N - 2];
                ro[N - 1] = ao[N - 1] = go[N - 1] = R(0);
#pragma unroll
                for (int v = N - 2; v >= 0; --v)
                    eliminate(v, v > 0 ? f[v - 1] : fp[N - 1], v > 0 ? gg[v - 1] : gp[N - 1], ro, ao, go);
                vF[swz(cc)] = V16<R>::pack(ro);
                vG[swz(cc)] = V16<R>::pack(ao);
                vQ[swz(cc)] = V16<R>::pack(go);
            }
            for (--cc; cc >= c_lo; --cc) {
#pragma unroll
                for (int v = 0; v < N; ++v) {
                    f[v] = fp[v];
                    gg[v] = gp[v];
                }
                load_prev(cc);
                R ro[N], ao[N], go[N];
#pragma unroll
                for (int v = N - 1; v >= 0; --v)
                    eliminate(v, v > 0 ? f[v - 1] : fp[N - 1], v > 0 ? gg[v - 1] : gp[N - 1], ro, ao, go);
                vF[swz(cc)] = V16<R>::pack(ro);
                vG[swz(cc)] = V16<R>::pack(ao);
                vQ[swz(cc)] = V16<R>::pack(go);
            }

            R X, Xm;
            if (P <= 32) {
                const int tn = (t + 1) & (P - 1);
                R rho_n = __shfl_sync(full, rho1, tn, P), alp_n = __shfl_sync(full, alp1, tn, P),
                  gam_n = __shfl_sync(full, gam1, tn, P);
                X = pcr_warp<R>(make_reduced<R>(ae, be, ce, re, qp, qq, qw, rho_n, alp_n, gam_n), t, P);
                Xm = __shfl_sync(full, X, (t - 1) & (P - 1), P);
            } else {
                R *small = reinterpret_cast<R *>(smem_raw + work_off) + LPB * LS + tm * 8 * P;
                small[t] = rho1;
                small[P + t] = alp1;
                small[2 * P + t] = gam1;
                __syncthreads();
                const int tn = (t + 1) & (P - 1);
                Reduced<R> q = make_reduced<R>(ae, be, ce, re, qp, qq, qw, small[tn], small[P + tn],
                                               small[2 * P + tn]);
                __syncthreads();
                X = pcr_smem<R>(q, t, P, small, small + P, small + 2 * P, small + 3 * P, 1);
                small[4 * P + t] = X;
                __syncthreads();
                Xm = small[4 * P + ((t - 1) & (P - 1))];
            }

            R dprev = Xm;
            for (int c2 = c_lo; c2 < c_hi - 1; ++c2) {
                R ro[N], ao[N], go[N], d[N];
                V16<R>::unpack(vF[swz(c2)], ro);
                V16<R>::unpack(vG[swz(c2)], ao);
                V16<R>::unpack(vQ[swz(c2)], go);
#pragma unroll
                for (int v = 0; v < N; ++v) {
                    d[v] = ro[v] - ao[v] * dprev - go[v] * X;
                    dprev = d[v];
                }
                vF[swz(c2)] = V16<R>::pack(d);
            }
            {
                const int c2 = c_hi - 1;
                R ro[N], ao[N], go[N], d[N];
                V16<R>::unpack(vF[swz(c2)], ro);
                V16<R>::unpack(vG[swz(c2)], ao);
                V16<R>::unpack(vQ[swz(c2)], go);
#pragma unroll
                for (int v = 0; v < N - 1; ++v) {
                    d[v] = ro[v] - ao[v] * dprev - go[v] * X;
                    dprev = d[v];
                }
                d[N - 1] = X;
                vF[swz(c2)] = V16<R>::pack(d);
            }
        }
        __syncthreads();

        // ---- C: T_new = T_old + delta (T_old re-read through L2: the staging
        // area already holds the next group's rows)
        if (!J.transpose_out) {
            if (active) {
                const VT *vo = reinterpret_cast<const VT *>(Tin + (size_t)lc * n);
                VT *out = reinterpret_cast<VT *>(static_cast<R *>(J.Tout) + (size_t)lc * n);
                for (int c = t; c < m; c += P) {
                    R to[N], d[N];
                    V16<R>::unpack(vo[c], to);
                    V16<R>::unpack(vF[swz(c)], d);
                    R sum = R(0);
#pragma unroll
                    for (int v = 0; v < N; ++v) {
                        to[v] += d[v];
                        sum += to[v];
                    }
                    bad |= !(fabs(sum) < R(INFINITY));
                    out[c] = V16<R>::pack(to);
                }
            }
        } else {
            // out[p][line] (position-major, nl wide): thread (group q4 of N lines,
            // position p), group fastest, reads the N deltas of position p (one
            // scalar per line, consecutive positions across lanes: no bank
            // conflicts) and T_old, and writes the N lines as one 16-byte store.
            R *out = static_cast<R *>(J.Tout);
            const int quads = LPB / N;  // a power of two in this mode
            const int logQ = __ffs(quads) - 1;
            const int q4 = threadIdx.x & (quads - 1);
            const int l0 = q4 * N;
            const R *src[N];
            const R *sl[N];
#pragma unroll
            for (int v = 0; v < N; ++v) {
                const int ln = line0 + l0 + v < nl ? line0 + l0 + v : nl - 1;
                src[v] = Tin + (size_t)ln * n;
                sl[v] = reinterpret_cast<R *>(smem_raw + work_off) + (l0 + v) * LS;
            }
            const bool vec_ok = (nl & (N - 1)) == 0 && line0 + l0 + N <= nl;
            const int pstride = blockDim.x >> logQ;
            for (int p = threadIdx.x >> logQ; p < n; p += pstride) {
                const int ap = at(p);
                R o[N];
                R sum = R(0);
#pragma unroll
                for (int v = 0; v < N; ++v) {
                    o[v] = src[v][p] + sl[v][ap];
                    sum += o[v];
                }
                bad |= !(fabs(sum) < R(INFINITY));
                R *dst = out + (size_t)p * nl + line0 + l0;
                if (vec_ok) {
                    *reinterpret_cast<VT *>(dst) = V16<R>::pack(o);
                } else {
#pragma unroll
                    for (int v = 0; v < N; ++v)
                        if (line0 + l0 + v < nl) dst[v] = o[v];
                }
            }
        }
        __syncthreads();  // working arrays and the job slot are reused by the next group
        cur ^= 1;
    }
    if (bad) atomicOr(args.err, 1u);
}

}  // namespace aniso
