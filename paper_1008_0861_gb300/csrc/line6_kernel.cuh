// line6_kernel.cuh -- long lines (2048 < n <= 4096 cells, FP32): the
// warp-autonomous line kernel's phases with a line's team spread over W
// warps (P = 32 W lanes), so that a block still holds four lines and the
// transposed store still writes 16-byte pieces.
//
// Same linear algebra and the same per-lane work as line4 (delta form,
// coalesced flux phase, bottom-up segment elimination in shared memory,
// reduced system of the segment-end unknowns, recovery, T_new = T_old +
// delta, transposed store).  What changes with a team wider than a warp:
//  - in the flux phase the cell after a lane's chunk comes from the next
//    lane by a shuffle inside the warp; the warp's last lane (whose next
//    chunk belongs to another warp, or to the next round) reads that cell's
//    three T values directly and forms its inner limited difference;
//  - the values a lane needs from its neighbours in the team (the flux of
//    the face below its segment, the next segment's first eliminated row,
//    the previous segment-end unknown) pass through shared memory between
//    block barriers, and the reduced system is solved by PCR in shared
//    memory (pcr_smem).
// Lines of the x-update are rows of T; of the y-update, rows of the
// column-major T*.  Each block holds `lines_per_block` lines; all lines of a
// launch have the same team size (block-wide barriers).
#pragma once
#include "line4_kernel.cuh"

namespace aniso {

template <typename C, bool VL>
__global__ void __launch_bounds__(512, 1) line6_kernel(Line2Args args)
{
    typedef float R;
    typedef float4 VT;
    constexpr int N = 4;
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
    const int W = P >> 5;  // warps per line
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lb = warp / W;               // line within the block
    const int t = (warp - lb * W) * 32 + lane;  // lane within the line's team
    const int line0 = (blockIdx.x - J.block0) * LPB;
    const int line = line0 + lb;
    const bool active = line < nl;
    const int lc = active ? line : nl - 1;
    int lu = lc + 1, ld = lc - 1;
    if (lu >= nl) lu = J.per_cross ? 0 : nl - 1;  // mirrored ghost line
    if (ld < 0) ld = J.per_cross ? nl - 1 : 0;
    const R *Tin = static_cast<const R *>(J.Tin);
    const R *rc = Tin + (size_t)lc * n, *ru = Tin + (size_t)lu * n, *rd = Tin + (size_t)ld * n;
    const C *G = static_cast<const C *>(J.g) + (size_t)lc * n;
    const C *E = static_cast<const C *>(J.e) + (size_t)lc * n;
    const R lam = (R)J.lam, mu = (R)J.mu;
    const unsigned full = 0xffffffffu;

    if (threadIdx.x == 0) {  // the block's rows into L2 (a hint)
        const int f0 = line0 > 0 ? line0 - 1 : line0, f1 = min(line0 + LPB + 1, nl), g1 = min(line0 + LPB, nl);
        l2_prefetch(Tin + (size_t)f0 * n, (size_t)(f1 - f0) * n * sizeof(R));
        l2_prefetch(static_cast<const C *>(J.g) + (size_t)line0 * n, (size_t)(g1 - line0) * n * sizeof(C));
        l2_prefetch(static_cast<const C *>(J.e) + (size_t)line0 * n, (size_t)(g1 - line0) * n * sizeof(C));
    }

    // segment of lane t: chunks [c_lo, c_lo + Ut); the first rr lanes one more
    const int U = m / P, rr = m % P;
    const int Ut = U + (t < rr ? 1 : 0);
    const int c_lo = t * U + (t < rr ? t : rr);
    const int V = U + (rr ? 1 : 0);  // chunk rounds of the coalesced phases
    const int mfull = m & ~7, logU = 31 - __clz(U);
    VT *sA = reinterpret_cast<VT *>(smem_raw) + (size_t)lb * 3 * m;  // F -> rho -> delta -> T_new
    VT *sB = sA + m;                                                  // lam*g -> alpha
    VT *sC = sA + 2 * m;                                              // gamma
    R *ex = reinterpret_cast<R *>(reinterpret_cast<VT *>(smem_raw) + (size_t)LPB * 3 * m) + (size_t)lb * 4 * P;
    R *ex0 = ex, *ex1 = ex + P, *ex2 = ex + 2 * P, *ex3 = ex + 3 * P;  // team exchange
    auto swz = [mfull, logU](int c) { return c < mfull ? c ^ ((c >> logU) & 7) : c; };

    // ---- A: face fluxes and lam*g, coalesced (lane t: chunks v*P + t), last
    // round first, with the loads of the next two rounds in flight.  The
    // cell after a chunk comes from the next lane by a shuffle; the warp's
    // last lane and the lane with the line's last chunk read it directly
    // (issued with the round's loads).
    {
        const VT *vd = reinterpret_cast<const VT *>(rd), *vc = reinterpret_cast<const VT *>(rc),
                 *vu = reinterpret_cast<const VT *>(ru);
        typedef decltype(ld_raw(G)) CT;
        struct In {
            VT c, d, u;
            CT g, e;
            R nc, nd, nu;  // T of the cell after the chunk (loaded where needed)
            int cur;
        };
        auto load = [&](int v) {
            In x;
            x.cur = min(v * P + t, m - 1);
            x.c = vc[x.cur];
            x.d = vd[x.cur];
            x.u = vu[x.cur];
            x.g = ld_raw(G + x.cur * N);
            x.e = ld_raw(E + x.cur * N);
            x.nc = x.nd = x.nu = R(0);
            if (lane == 31 || x.cur == m - 1) {
                const int p1 = x.cur == m - 1 ? (J.per_line ? 0 : n - 1) : N * (x.cur + 1);
                x.nc = rc[p1];
                x.nd = rd[p1];
                x.nu = ru[p1];
            }
            return x;
        };
        In cur = load(V - 1);
        In nxt = V >= 2 ? load(V - 2) : cur;
        for (int v = V - 1; v >= 0; --v) {
            const In x = cur;
            cur = nxt;
            if (v >= 2) nxt = load(v - 2);
            const int c = v * P + t;
            R Td[N], Tc[N], Tu[N], Gv[N], Ev[N];
            V16<R>::unpack(x.c, Tc);
            V16<R>::unpack(x.d, Td);
            V16<R>::unpack(x.u, Tu);
            unpack_raw(x.g, Gv);
            unpack_raw(x.e, Ev);
            R vv[N];
#pragma unroll
            for (int j = 0; j < N; ++j) vv[j] = level<R, VL>(lim, Tu[j] - Tc[j], Tc[j] - Td[j]);
            R nT = __shfl_down_sync(full, Tc[0], 1), nv = __shfl_down_sync(full, vv[0], 1);
            if (lane == 31 || x.cur == m - 1) {
                nT = x.nc;
                nv = level<R, VL>(lim, x.nu - nT, nT - x.nd);
            }
            R F[N], lg[N];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const R Tnx = j + 1 < N ? Tc[j + 1] : nT;
                const R vnx = j + 1 < N ? vv[j + 1] : nv;
                lg[j] = lam * Gv[j];
                F[j] = lg[j] * (Tnx - Tc[j]) + mu * Ev[j] * level<R, VL>(lim, vv[j], vnx);
            }
            if (c < m) {
                sA[swz(c)] = V16<R>::pack(F);
                sB[swz(c)] = V16<R>::pack(lg);
            }
        }
    }
    __syncthreads();

    // ---- B1: bottom-up elimination of lane t's segment
    R rho1 = R(0), alp1 = R(0), gam1 = R(-1);
    R qp = R(0), qq = R(1), qw = R(0);
    R ae = R(0), be = R(1), ce = R(0), re = R(0);
    R Fpend = R(0), lgpend = R(0), Flast = R(0), lglast = R(0);
    R ro[N], ao[N], go[N];  // maps of the chunk above, waiting for its row 0
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
    {
#pragma unroll
        for (int v = 0; v < N; ++v) ro[v] = ao[v] = go[v] = R(0);
        for (int u = Ut - 1; u >= 0; --u) {
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
                sC[swz(c + 1)] = V16<R>::pack(go);
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
    }
    // row s needs the face below the segment: the previous lane's last face
    ex0[t] = Flast;
    ex1[t] = lglast;
    __syncthreads();
    {
        const int tp = (t - 1 + P) % P;
        elim(Fpend, ex0[tp], lgpend, ex1[tp], ro[0], ao[0], go[0]);
        sA[swz(c_lo)] = V16<R>::pack(ro);
        sB[swz(c_lo)] = V16<R>::pack(ao);
        sC[swz(c_lo)] = V16<R>::pack(go);
    }
    __syncthreads();

    // Phase C's first two chunks of T_old start loading now.
    const VT *vcC = reinterpret_cast<const VT *>(rc);
    VT pre0 = vcC[t < m ? t : m - 1], pre1 = pre0;
    if (t + P < m) pre1 = vcC[t + P];

    // ---- R: reduced system of the line in the segment-end unknowns
    R X, Xm;
    {
        ex0[t] = rho1;
        ex1[t] = alp1;
        ex2[t] = gam1;
        __syncthreads();
        const int tn = (t + 1) % P;
        const R rho_n = ex0[tn], alp_n = ex1[tn], gam_n = ex2[tn];
        __syncthreads();
        X = pcr_smem<R>(make_reduced<R>(ae, be, ce, re, qp, qq, qw, rho_n, alp_n, gam_n), t, P, ex0, ex1, ex2,
                        ex3, 1);
        ex0[t] = X;
        __syncthreads();
        Xm = ex0[(t - 1 + P) % P];
    }

    // ---- B2: forward recovery of lane t's segment (delta over rho)
    {
        R dprev = Xm;
        for (int u = 0; u < Ut; ++u) {
            const int c = c_lo + u;
            R r4[N], a4[N], g4[N], d[N];
            V16<R>::unpack(sA[swz(c)], r4);
            V16<R>::unpack(sB[swz(c)], a4);
            V16<R>::unpack(sC[swz(c)], g4);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                d[j] = (u == Ut - 1 && j == N - 1) ? X : r4[j] - a4[j] * dprev - g4[j] * X;
                dprev = d[j];
            }
            sA[swz(c)] = V16<R>::pack(d);
        }
    }
    __syncthreads();

    // ---- C: T_new = T_old + delta, coalesced; staged for the store
    bool bad = false;
    for (int v = 0; v < V; ++v) {
        const int c = v * P + t;
        if (c >= m) break;
        R to[N], d[N];
        V16<R>::unpack(pre0, to);
        pre0 = pre1;
        if (c + 2 * P < m) pre1 = vcC[c + 2 * P];
        V16<R>::unpack(sA[swz(c)], d);
        R sum = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            to[j] += d[j];
            sum += to[j];
        }
        bad |= !(fabsf(sum) < INFINITY);
        if (!J.transpose_out) {
            if (active) reinterpret_cast<VT *>(static_cast<R *>(J.Tout) + (size_t)lc * n)[c] = V16<R>::pack(to);
        } else {
            sA[swz(c)] = V16<R>::pack(to);
        }
    }

    // ---- transposed store: out[p][line], the block's lines in 16-byte pieces
    if (J.transpose_out) {
        __syncthreads();
        R *out = static_cast<R *>(J.Tout);
        const int groups = LPB >> 2;
        const bool vec_ok = (nl & 3) == 0;
        if (LPB == 2) {  // two lines: 8-byte pieces
            for (int p = threadIdx.x; p < n; p += blockDim.x) {
                const int sc = swz(p >> 2), j = p & 3;
                const R o0 = reinterpret_cast<const R *>(reinterpret_cast<const VT *>(smem_raw) + sc)[j];
                const R o1 = reinterpret_cast<const R *>(reinterpret_cast<const VT *>(smem_raw) + 3 * m + sc)[j];
                R *dst = out + (size_t)p * nl + line0;
                if ((nl & 1) == 0 && line0 + 2 <= nl) {
                    *reinterpret_cast<float2 *>(dst) = make_float2(o0, o1);
                } else {
                    if (line0 < nl) dst[0] = o0;
                    if (line0 + 1 < nl) dst[1] = o1;
                }
            }
        }
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int sc = swz(p >> 2), j = p & 3;
            for (int grp = 0; grp < groups; ++grp) {
                R o[N];
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const int l = (grp << 2) + i;
                    o[i] = reinterpret_cast<const R *>(reinterpret_cast<const VT *>(smem_raw) + (size_t)l * 3 * m + sc)[j];
                }
                const int l0 = line0 + (grp << 2);
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
}

}  // namespace aniso
