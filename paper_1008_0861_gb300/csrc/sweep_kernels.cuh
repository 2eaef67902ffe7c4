// sweep_kernels.cuh -- device code for one directional update of the split
// semi-implicit scheme (Sharma & Hammett, arXiv:1008.0861, Section 2).
//
// Both updates solve, for every grid line, the tridiagonal system of
// Eq. xup (rows) or Eq. yup (columns).  Written in delta form, with
// delta = T_new - T_old and face p+1/2 carrying the flux
//     F_p = lam g_p (T_{p+1} - T_p) + mu e_p DeltaTbar_p,
// the line system is
//     -lam g_{p-1} delta_{p-1} + (1 + lam (g_{p-1} + g_p)) delta_p
//         - lam g_p delta_{p+1} = F_p - F_{p-1},
// which is Eq. xup / Eq. yup with T_old moved to the right-hand side:
// g is the normal coefficient (b-bar_x^2 or b-bar_y^2), e the transverse
// coefficient (b-bar_x b-bar_y), DeltaTbar the limited transverse difference
// (the DeltaT-bar equations after Eq. yup, limiter of Eq. vanLeer).
//
// Line solve (no counterpart in the paper, which only notes that the line
// systems can be solved directly and cheaply): each line is cut into P segments, one
// per thread.  A thread eliminates its segment bottom-up, storing
//     delta_k = rho_k - alpha_k delta_{k-1} - gamma_k delta_e       (s <= k < e)
// and composing those maps into delta_{e-1} = p + q delta_{s-1} + w delta_e.
// Substituting into row e and the next segment's first map gives one
// equation per segment in the segment-end unknowns X_t = delta_{e_t}:
//     L_t X_{t-1} + D_t X_t + U_t X_{t+1} = R_t,
// a (cyclic when periodic) tridiagonal system of size P, solved by parallel
// cyclic reduction with indices taken mod P (P is a power of two, so the
// zero corner entries of a non-periodic system stay zero).  A forward pass
// then recovers every delta_k.  All pivots are >= 1 because each line matrix
// is a strictly diagonally dominant M-matrix.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "aniso_internal.h"

namespace aniso {

// ------------------------------------------------------------ arithmetic

template <typename R> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
};

__device__ __forceinline__ float ldcoef(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ldcoef(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldcoef(const __half *p) { return __half2float(__ldg(p)); }

template <typename R> __device__ __forceinline__ bool same_sign(R a, R b)
{
    return (a > R(0) && b > R(0)) || (a < R(0) && b < R(0));
}

// Two-argument limiters (Eq. vanLeer; minmod and MC as named in Section 2).
template <typename R> __device__ __forceinline__ R lim2(int lim, R a, R b)
{
    if (!same_sign(a, b)) return R(0);
    if (lim == LIM_VANLEER) return Num<R>::div(R(2) * a * b, a + b);
    if (lim == LIM_MINMOD) return a > R(0) ? fmin(a, b) : fmax(a, b);
    R m = fmin(fmin(R(2) * fabs(a), R(2) * fabs(b)), R(0.5) * fabs(a + b));
    return a > R(0) ? m : -m;
}

// L(a,b,c,d) = L(L(a,b), L(c,d)); the arithmetic mean for LIM_ARITH.
template <typename R> __device__ __forceinline__ R limit4(int lim, R a, R b, R c, R d)
{
    if (lim == LIM_ARITH) return R(0.25) * (a + b + c + d);
    return lim2<R>(lim, lim2<R>(lim, a, b), lim2<R>(lim, c, d));
}

// Face flux through face p+1/2 of a line from the cells on both sides of
// the face (c0 = this line, u/d = the lines after/before it across).
template <typename R>
__device__ __forceinline__ R face_flux(int lim, R lam, R mu, R g, R e, R d0, R c0, R u0, R d1, R c1,
                                       R u1)
{
    R dT = limit4<R>(lim, u1 - c1, c1 - d1, u0 - c0, c0 - d0);
    return lam * g * (c1 - c0) + mu * e * dT;
}

// Compensated state (Kahan, FP32): a cell holds hi + lo.  Differences of two
// cells are formed as (hi_a - hi_b) + (lo_a - lo_b); with K = false lo is 0
// and the expressions reduce to plain differences.
template <typename R, bool K> __device__ __forceinline__ R dif(R ah, R al, R bh, R bl)
{
    return K ? (ah - bh) + (al - bl) : ah - bh;
}
template <typename R, bool K>
__device__ __forceinline__ R face_flux_k(int lim, R lam, R mu, R g, R e, R d0h, R d0l, R c0h, R c0l, R u0h,
                                         R u0l, R d1h, R d1l, R c1h, R c1l, R u1h, R u1l)
{
    const R dT = limit4<R>(lim, dif<R, K>(u1h, u1l, c1h, c1l), dif<R, K>(c1h, c1l, d1h, d1l),
                           dif<R, K>(u0h, u0l, c0h, c0l), dif<R, K>(c0h, c0l, d0h, d0l));
    return lam * g * dif<R, K>(c1h, c1l, c0h, c0l) + mu * e * dT;
}
// FP64 value -> (hi, lo) float pair (hi + lo reproduces it to ~48 bits).
__device__ __forceinline__ void split_f64(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}
__device__ __forceinline__ void split_f64(double v, double &hi, double &lo)
{
    hi = v;
    lo = 0.0;
}

// (hi, lo) + d with an exact two-sum of hi + d, the rounding error folded
// into lo and the pair renormalised.
template <typename R>
__device__ __forceinline__ void kahan_add(R hi, R lo, R d, R &ohi, R &olo)
{
    const R s = hi + d;
    const R bb = s - hi;
    const R err = (hi - (s - bb)) + (d - bb);
    const R l2 = lo + err;
    const R h2 = s + l2;
    olo = l2 - (h2 - s);
    ohi = h2;
}

// Error-free transformations (Knuth's TwoSum; Dekker's FastTwoSum, |a| >= |b|):
// a + b == s + e exactly in the working precision.
template <typename R> __device__ __forceinline__ void two_sum(R a, R b, R &s, R &e)
{
    s = a + b;
    const R bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
template <typename R> __device__ __forceinline__ void fast_two_sum(R a, R b, R &s, R &e)
{
    s = a + b;
    e = b - (s - a);
}
// Compensated accumulator: the running sum is s + c.
template <typename R> struct CSum {
    R s = R(0), c = R(0);
    __device__ __forceinline__ void add(R x)
    {
        R t, e;
        two_sum(s, x, t, e);
        s = t;
        c += e;
    }
};
// (hi, lo) + (d - corr), corr = ch + cl, in double-word arithmetic of the
// working precision (relative error of order 2^-2p): d - corr as an exact
// pair, then the pair sum renormalised so that |ol| <= ulp(oh)/2.
template <typename R>
__device__ __forceinline__ void dw_update(R hi, R lo, R d, R ch, R cl, R &oh, R &ol)
{
    R dh, dl;
    two_sum(d, -ch, dh, dl);
    dl -= cl;
    R sh, se;
    two_sum(hi, dh, sh, se);
    se += lo + dl;
    fast_two_sum(sh, se, oh, ol);
}

// Padded shared-memory index: one spare word per 32 keeps threads that walk
// neighbouring segments on different banks.
__device__ __forceinline__ int phys(int k) { return k + (k >> 5); }

// -------------------------------------------- reduced system of one line
//
// Inputs per thread t of a team: row e of its segment (ae, be, ce, re), its
// composite map (qp, qq, qw) and its top map (rho, alpha, gamma at k = s).
// Output: X_t = delta at the segment's last cell, and X_{t-1}.

template <typename R> struct Reduced {
    R L, D, U, Rr;
};

template <typename R>
__device__ __forceinline__ Reduced<R> make_reduced(R ae, R be, R ce, R re, R qp, R qq, R qw,
                                                   R rho_n, R alp_n, R gam_n)
{
    Reduced<R> r;
    r.L = ae * qq;
    r.D = be + ae * qw - ce * alp_n;
    r.U = -ce * gam_n;
    r.Rr = re - ae * qp - ce * rho_n;
    return r;
}

// PCR for a team of P <= 32 consecutive lanes (width-P shuffles).
template <typename R> __device__ __forceinline__ R pcr_warp(Reduced<R> q, int t, int P)
{
    const unsigned full = 0xffffffffu;
    for (int h = 1; h < P; h <<= 1) {
        int tm = (t - h) & (P - 1), tp = (t + h) & (P - 1);
        R Lm = __shfl_sync(full, q.L, tm, P), Dm = __shfl_sync(full, q.D, tm, P);
        R Um = __shfl_sync(full, q.U, tm, P), Rm = __shfl_sync(full, q.Rr, tm, P);
        R Lp = __shfl_sync(full, q.L, tp, P), Dp = __shfl_sync(full, q.D, tp, P);
        R Up = __shfl_sync(full, q.U, tp, P), Rp = __shfl_sync(full, q.Rr, tp, P);
        R k1 = Num<R>::div(q.L, Dm), k2 = Num<R>::div(q.U, Dp);
        q.D = q.D - k1 * Um - k2 * Lp;
        q.Rr = q.Rr - k1 * Rm - k2 * Rp;
        q.L = -k1 * Lm;
        q.U = -k2 * Up;
    }
    return Num<R>::div(q.Rr, q.L + q.D + q.U);
}

// PCR through shared memory: element t of the system lives at buf[t*stride];
// all threads of the block must call it the same number of times.
template <typename R>
__device__ __forceinline__ R pcr_smem(Reduced<R> q, int t, int P, R *sL, R *sD, R *sU, R *sR,
                                      int stride)
{
    for (int h = 1; h < P; h <<= 1) {
        sL[t * stride] = q.L;
        sD[t * stride] = q.D;
        sU[t * stride] = q.U;
        sR[t * stride] = q.Rr;
        __syncthreads();
        int tm = ((t - h) & (P - 1)) * stride, tp = ((t + h) & (P - 1)) * stride;
        R k1 = Num<R>::div(q.L, sD[tm]), k2 = Num<R>::div(q.U, sD[tp]);
        R nD = q.D - k1 * sU[tm] - k2 * sL[tp];
        R nR = q.Rr - k1 * sR[tm] - k2 * sR[tp];
        R nL = -k1 * sL[tm];
        R nU = -k2 * sU[tp];
        __syncthreads();
        q.L = nL;
        q.U = nU;
        q.D = nD;
        q.Rr = nR;
    }
    return Num<R>::div(q.Rr, q.L + q.D + q.U);
}

__device__ __forceinline__ void flag_nonfinite(unsigned *err, float v)
{
    if (!isfinite(v)) atomicOr(err, 1u);
}
__device__ __forceinline__ void flag_nonfinite(unsigned *err, double v)
{
    if (!isfinite(v)) atomicOr(err, 1u);
}

// Find the job that owns this block (jobs sorted by block0).
template <typename Job> __device__ __forceinline__ int find_job(const Job *jobs, int njobs)
{
    int b = blockIdx.x, lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block0 <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ====================================================== contiguous lines
//
// Rows of Eq. xup (and columns of Eq. yup on a transposed grid).  Phases:
//  A  coalesced: face fluxes F_p and normal coefficients g_p -> shared memory
//  B1 per segment: bottom-up elimination, maps stored in shared memory
//  R  reduced system of the line (PCR)
//  B2 per segment: forward recovery of delta
//  C  coalesced: T_new = T_old + delta

template <typename R, typename C, bool K>
__global__ void __launch_bounds__(512) line_sweep_kernel(LineArgs args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_job;
    if (args.jobs) {
        if (threadIdx.x == 0) s_job = find_job(args.jobs, args.njobs);
        __syncthreads();
    }
    const LineJob J = args.jobs ? args.jobs[s_job] : args.one;
    const int lim = args.limiter;
    const int P = J.team, n = J.n;
    const int tm = threadIdx.x / P, t = threadIdx.x - tm * P;
    const int line = (blockIdx.x - J.block0) * J.lines_per_block + tm;
    const bool active = line < J.nlines;
    const int lc = active ? line : J.nlines - 1;
    int lu = lc + 1, ld = lc - 1;
    if (lu >= J.nlines) lu = J.per_cross ? 0 : J.nlines - 1;  // mirrored ghost line
    if (ld < 0) ld = J.per_cross ? J.nlines - 1 : 0;
    const R *Tin = static_cast<const R *>(J.Tin);
    const R *rc = Tin + (size_t)lc * n, *ru = Tin + (size_t)lu * n, *rd = Tin + (size_t)ld * n;
    // low parts of the compensated state (K only)
    const R *TinL = static_cast<const R *>(J.TinLo);
    const R *rcl = K ? TinL + (size_t)lc * n : nullptr, *rul = K ? TinL + (size_t)lu * n : nullptr,
            *rdl = K ? TinL + (size_t)ld * n : nullptr;
    const C *G = static_cast<const C *>(J.g) + (size_t)lc * n;
    const C *E = static_cast<const C *>(J.e) + (size_t)lc * n;
    const R lam = (R)J.lam, mu = (R)J.mu;

    const int np = n + (n >> 5) + 1;
    R *sF = reinterpret_cast<R *>(smem_raw) + (size_t)tm * 3 * np;  // F, then rho, then delta
    R *sG = sF + np;                                                  // g, then alpha
    R *sQ = sG + np;                                                  // gamma
    R *small = reinterpret_cast<R *>(smem_raw) + (size_t)J.lines_per_block * 3 * np +
               (size_t)tm * 8 * P;

    // ---- A: fluxes through every face p+1/2 of the line.  Batches of UA
    // cells per thread issue all their loads before any arithmetic so that
    // many loads are in flight; the value at p+1 comes from the neighbouring
    // lane (the last lane of each width-wide group loads it).
    {
        constexpr int UA = 4;
        const int width = P < 32 ? P : 32;
        const int lane_in = t & (width - 1);
        const unsigned full = 0xffffffffu;
        for (int p0 = t; p0 - t < n; p0 += UA * P) {
            R vd[UA], vc[UA], vu[UA], vg[UA], ve[UA];
            R wd[UA] = {}, wc[UA] = {}, wu[UA] = {};  // low parts (K only)
#pragma unroll
            for (int u = 0; u < UA; ++u) {
                const int p = p0 + u * P;
                const int pc = p < n ? p : n - 1;
                vd[u] = rd[pc];
                vc[u] = rc[pc];
                vu[u] = ru[pc];
                if (K) {
                    wd[u] = rdl[pc];
                    wc[u] = rcl[pc];
                    wu[u] = rul[pc];
                }
                vg[u] = ldcoef(G + pc);
                ve[u] = ldcoef(E + pc);
            }
#pragma unroll
            for (int u = 0; u < UA; ++u) {
                const int p = p0 + u * P;
                R vd1 = __shfl_down_sync(full, vd[u], 1, width);
                R vc1 = __shfl_down_sync(full, vc[u], 1, width);
                R vu1 = __shfl_down_sync(full, vu[u], 1, width);
                R wd1 = R(0), wc1 = R(0), wu1 = R(0);
                if (K) {
                    wd1 = __shfl_down_sync(full, wd[u], 1, width);
                    wc1 = __shfl_down_sync(full, wc[u], 1, width);
                    wu1 = __shfl_down_sync(full, wu[u], 1, width);
                }
                if (p < n) {
                    int p1 = p + 1;
                    if (lane_in == width - 1 || p1 >= n) {
                        if (p1 == n) p1 = J.per_line ? 0 : n - 1;
                        vd1 = rd[p1];
                        vc1 = rc[p1];
                        vu1 = ru[p1];
                        if (K) {
                            wd1 = rdl[p1];
                            wc1 = rcl[p1];
                            wu1 = rul[p1];
                        }
                    }
                    sF[phys(p)] = face_flux_k<R, K>(lim, lam, mu, vg[u], ve[u], vd[u], wd[u], vc[u], wc[u],
                                                    vu[u], wu[u], vd1, wd1, vc1, wc1, vu1, wu1);
                    sG[phys(p)] = vg[u];
                }
            }
        }
    }
    __syncthreads();

    // ---- B1: segment [s, e], bottom-up elimination
    const int s = (int)(((long long)t * n) / P), e = (int)(((long long)(t + 1) * n) / P) - 1;
    const int em1 = e - 1 < 0 ? e - 1 + n : e - 1;
    const R ge = sG[phys(e)], gem = sG[phys(em1)];
    // fixed boundary nodes: identity rows (delta = 0) for the line's end cells,
    // or for every cell of a fixed line
    const bool ident = J.pin_lines && (lc == 0 || lc == J.nlines - 1);
    const bool pin_e = ident || (J.pin_ends && (e == 0 || e == n - 1));
    const R re = pin_e ? R(0) : sF[phys(e)] - sF[phys(em1)];
    const R ae = pin_e ? R(0) : -lam * gem, ce = pin_e ? R(0) : -lam * ge, be = R(1) - ae - ce;
    R rho1 = R(0), alp1 = R(0), gam1 = R(-1);  // map of the virtual row e: delta_e = delta_e
    R qp = R(0), qq = R(1), qw = R(0);          // composite map, starts as the identity
    R gk = gem, Fk = sF[phys(em1)];  // values at k = e-1, carried down the loop
    for (int k = e - 1; k >= s; --k) {
        const int km = k - 1 < 0 ? k - 1 + n : k - 1;
        const R gkm = sG[phys(km)], Fkm = sF[phys(km)];
        const bool pin_k = ident || (J.pin_ends && k == 0);
        const R rk = pin_k ? R(0) : Fk - Fkm;
        const R a = pin_k ? R(0) : -lam * gkm, c = pin_k ? R(0) : -lam * gk, b = R(1) - a - c;
        gk = gkm;
        Fk = Fkm;
        const R inv = Num<R>::div(R(1), b - c * alp1);
        const R alp = a * inv, gam = -c * gam1 * inv, rho = (rk - c * rho1) * inv;
        sF[phys(k)] = rho;
        sG[phys(k)] = alp;
        sQ[phys(k)] = gam;
        qp = qp + qq * rho;
        qw = qw - qq * gam;
        qq = -qq * alp;
        rho1 = rho;
        alp1 = alp;
        gam1 = gam;
    }

    // ---- R: reduced system in the segment-end unknowns
    R X, Xm;
    if (P <= 32) {
        const unsigned full = 0xffffffffu;
        const int tn = (t + 1) & (P - 1);
        R rho_n = __shfl_sync(full, rho1, tn, P), alp_n = __shfl_sync(full, alp1, tn, P),
          gam_n = __shfl_sync(full, gam1, tn, P);
        X = pcr_warp<R>(make_reduced<R>(ae, be, ce, re, qp, qq, qw, rho_n, alp_n, gam_n), t, P);
        Xm = __shfl_sync(full, X, (t - 1) & (P - 1), P);
    } else {
        R *sTop = small;  // [3][P]
        sTop[t] = rho1;
        sTop[P + t] = alp1;
        sTop[2 * P + t] = gam1;
        __syncthreads();
        const int tn = (t + 1) & (P - 1);
        Reduced<R> q = make_reduced<R>(ae, be, ce, re, qp, qq, qw, sTop[tn], sTop[P + tn],
                                       sTop[2 * P + tn]);
        __syncthreads();
        R *sL = small, *sD = small + P, *sU = small + 2 * P, *sRr = small + 3 * P;
        X = pcr_smem<R>(q, t, P, sL, sD, sU, sRr, 1);
        R *sX = small + 4 * P;
        sX[t] = X;
        __syncthreads();
        Xm = sX[(t - 1) & (P - 1)];
    }

    // ---- B2: forward recovery
    {
        R dprev = Xm;
        for (int k = s; k < e; ++k) {
            const R d = sF[phys(k)] - sG[phys(k)] * dprev - sQ[phys(k)] * X;
            sF[phys(k)] = d;
            dprev = d;
        }
        sF[phys(e)] = X;
    }
    __syncthreads();

    // ---- C: T_new = T_old + delta.
    // Compensated state: in exact arithmetic every line's sum of delta is zero
    // (the right-hand side telescopes and each line matrix has unit column
    // sums), so the line's compensated sum of the computed delta is rounding
    // residual; it is removed evenly and hi + lo + delta - corr is formed in
    // double-word FP32 arithmetic, which conserves the sum of hi + lo across
    // the update to far below FP32 rounding.  FP64 only combines the threads'
    // partial sums (a few operations per thread, none per cell).
    if (K) {
        CSum<R> acc;
        for (int p = t; p < n; p += P) acc.add(sF[phys(p)]);
        double part = (double)acc.s + (double)acc.c;
        double lsum;
        if (P <= 32) {
            for (int o = 1; o < P; o <<= 1) part += __shfl_xor_sync(0xffffffffu, part, o, P);
            lsum = part;
        } else {
            // PCR area (8P floats), free now; rounded up to an 8-byte boundary
            double *red = reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(small) + 7) & ~uintptr_t(7));
            red[t] = part;
            __syncthreads();
            if (t == 0) {
                double a = 0.0;
                for (int k = 0; k < P; ++k) a += red[k];
                red[P] = a;
            }
            __syncthreads();
            lsum = red[P];
        }
        R ch, cl;
        split_f64(lsum / (double)n, ch, cl);
        if (active) {
            R *out = static_cast<R *>(J.Tout) + (size_t)lc * n;
            R *outl = static_cast<R *>(J.ToutLo) + (size_t)lc * n;
            for (int p = t; p < n; p += P) {
                R hi, lo;
                dw_update(rc[p], rcl[p], sF[phys(p)], ch, cl, hi, lo);
                out[p] = hi;
                outl[p] = lo;
                flag_nonfinite(args.err, hi);
            }
        }
    } else if (active) {
        constexpr int UC = 8;
        R *out = static_cast<R *>(J.Tout) + (size_t)lc * n;
        for (int p0 = t; p0 < n; p0 += UC * P) {
            R vo[UC], wo[UC] = {};
#pragma unroll
            for (int u = 0; u < UC; ++u) {
                const int p = p0 + u * P;
                vo[u] = p < n ? rc[p] : R(0);
                if (K) wo[u] = p < n ? rcl[p] : R(0);
            }
#pragma unroll
            for (int u = 0; u < UC; ++u) {
                const int p = p0 + u * P;
                if (p < n) {
                    if (K) {
                        R hi, lo;
                        kahan_add(vo[u], wo[u], sF[phys(p)], hi, lo);
                        out[p] = hi;
                        static_cast<R *>(J.ToutLo)[(size_t)lc * n + p] = lo;
                        flag_nonfinite(args.err, hi);
                    } else {
                        const R v = vo[u] + sF[phys(p)];
                        out[p] = v;
                        flag_nonfinite(args.err, v);
                    }
                }
            }
        }
    }
}

// ================================================== columns, row-major
//
// Eq. yup in the natural layout: a block owns Wb adjacent columns and all
// ny rows; thread (c, t) walks rows of segment t of column c, so every
// global access is coalesced across c.  Pass B1 reads the grid directly,
// bottom-up, and keeps the segment maps in shared memory.

template <typename R, typename C, bool K>
__global__ void __launch_bounds__(512) col_sweep_kernel(ColArgs args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_job;
    if (args.jobs) {
        if (threadIdx.x == 0) s_job = find_job(args.jobs, args.njobs);
        __syncthreads();
    }
    const ColJob J = args.jobs ? args.jobs[s_job] : args.one;
    const int lim = args.limiter;
    const int P = J.P, Wb = J.Wb, nx = J.nx, ny = J.ny;
    const int c = threadIdx.x % Wb, t = threadIdx.x / Wb;
    const int i = (blockIdx.x - J.block0) * Wb + c;
    const bool active = i < nx;
    const int ic = active ? i : nx - 1;
    int il = ic - 1, ir = ic + 1;
    if (il < 0) il = J.per_x ? nx - 1 : 0;  // mirrored ghost column
    if (ir >= nx) ir = J.per_x ? 0 : nx - 1;
    const R *Tin = static_cast<const R *>(J.Tin);
    const C *Gc = static_cast<const C *>(J.g);
    const C *Ec = static_cast<const C *>(J.e);
    const R lam = (R)J.lam, mu = (R)J.mu;
    const int s = (int)(((long long)t * ny) / P), e = (int)(((long long)(t + 1) * ny) / P) - 1;

    const int rows = ny + P;
    R *sRho = reinterpret_cast<R *>(smem_raw);
    R *sAlp = sRho + (size_t)rows * Wb;
    R *sGam = sAlp + (size_t)rows * Wb;
    R *small = sGam + (size_t)rows * Wb;  // 8 * P * Wb
    auto ph = [&](int k) { return (k + t) * Wb + c; };  // one spare row per segment
    auto rowmap = [&](int k) {
        if (k < 0) return J.per_y ? k + ny : 0;
        if (k >= ny) return J.per_y ? k - ny : ny - 1;
        return k;
    };

    const R *TinL = static_cast<const R *>(J.TinLo);  // low parts (K only)
    // row k: values (hi h, lo w) of columns i-1, i, i+1
    R l0, m0, r0, l1, m1, r1;
    R lw0 = 0, mw0 = 0, rw0 = 0, lw1 = 0, mw1 = 0, rw1 = 0;
    {
        const size_t o1 = (size_t)rowmap(e + 1) * nx, o0 = (size_t)e * nx;
        l1 = Tin[o1 + il];
        m1 = Tin[o1 + ic];
        r1 = Tin[o1 + ir];
        l0 = Tin[o0 + il];
        m0 = Tin[o0 + ic];
        r0 = Tin[o0 + ir];
        if (K) {
            lw1 = TinL[o1 + il];
            mw1 = TinL[o1 + ic];
            rw1 = TinL[o1 + ir];
            lw0 = TinL[o0 + il];
            mw0 = TinL[o0 + ic];
            rw0 = TinL[o0 + ir];
        }
    }
    // F_e: face e+1/2 (coefficient index e; the boundary face is zero under zero-flux)
    R ge = ldcoef(Gc + (size_t)e * nx + ic);
    R Fk = face_flux_k<R, K>(lim, lam, mu, ge, ldcoef(Ec + (size_t)e * nx + ic), l0, lw0, m0, mw0, r0, rw0,
                             l1, lw1, m1, mw1, r1, rw1);
    R gk = ge;
    // row e: needs F_{e-1} and g_{e-1}
    R ae, be, ce, re;
    {
        const int km = e - 1, kf = km < 0 ? km + ny : km;
        const size_t om = (size_t)rowmap(km) * nx;
        R lm = Tin[om + il], mm = Tin[om + ic], rm = Tin[om + ir];
        R lwm = 0, mwm = 0, rwm = 0;
        if (K) {
            lwm = TinL[om + il];
            mwm = TinL[om + ic];
            rwm = TinL[om + ir];
        }
        R gkm = ldcoef(Gc + (size_t)kf * nx + ic);
        R Fkm = face_flux_k<R, K>(lim, lam, mu, gkm, ldcoef(Ec + (size_t)kf * nx + ic), lm, lwm, mm, mwm, rm,
                                  rwm, l0, lw0, m0, mw0, r0, rw0);
        re = Fk - Fkm;
        ae = -lam * gkm;
        ce = -lam * gk;
        be = R(1) - ae - ce;
        Fk = Fkm;
        gk = gkm;
        l0 = lm;
        m0 = mm;
        r0 = rm;
        lw0 = lwm;
        mw0 = mwm;
        rw0 = rwm;
    }
    R rho1 = R(0), alp1 = R(0), gam1 = R(-1);
    R qp = R(0), qq = R(1), qw = R(0);
    // Rows are fetched UB at a time (all loads of a batch issued before the
    // elimination consumes them) so that each thread keeps many loads in flight.
    constexpr int UB = sizeof(R) == 8 ? 4 : 8;
    for (int k0 = e - 1; k0 >= s; k0 -= UB) {
        R Lv[UB], Mv[UB], Rv[UB], Gv[UB], Ev[UB];
        R Lw[UB] = {}, Mw[UB] = {}, Rw[UB] = {};
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int k = k0 - u >= s ? k0 - u : s;  // tail of the segment: repeat a valid row
            const int km = k - 1, kf = km < 0 ? km + ny : km;
            const size_t om = (size_t)rowmap(km) * nx;
            Lv[u] = Tin[om + il];
            Mv[u] = Tin[om + ic];
            Rv[u] = Tin[om + ir];
            if (K) {
                Lw[u] = TinL[om + il];
                Mw[u] = TinL[om + ic];
                Rw[u] = TinL[om + ir];
            }
            Gv[u] = ldcoef(Gc + (size_t)kf * nx + ic);
            Ev[u] = ldcoef(Ec + (size_t)kf * nx + ic);
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int k = k0 - u;
            if (k < s) break;
            const R gkm = Gv[u];
            const R Fkm = face_flux_k<R, K>(lim, lam, mu, gkm, Ev[u], Lv[u], Lw[u], Mv[u], Mw[u], Rv[u], Rw[u],
                                            l0, lw0, m0, mw0, r0, rw0);
            const R rk = Fk - Fkm;
            const R a = -lam * gkm, cc = -lam * gk, b = R(1) - a - cc;
            const R inv = Num<R>::div(R(1), b - cc * alp1);
            const R alp = a * inv, gam = -cc * gam1 * inv, rho = (rk - cc * rho1) * inv;
            sRho[ph(k)] = rho;
            sAlp[ph(k)] = alp;
            sGam[ph(k)] = gam;
            qp = qp + qq * rho;
            qw = qw - qq * gam;
            qq = -qq * alp;
            rho1 = rho;
            alp1 = alp;
            gam1 = gam;
            Fk = Fkm;
            gk = gkm;
            l0 = Lv[u];
            m0 = Mv[u];
            r0 = Rv[u];
            lw0 = Lw[u];
            mw0 = Mw[u];
            rw0 = Rw[u];
        }
    }

    // reduced system of column c across its P segments (threads t*Wb + c)
    R *sTop = small;  // [3][P][Wb]
    sTop[(0 * P + t) * Wb + c] = rho1;
    sTop[(1 * P + t) * Wb + c] = alp1;
    sTop[(2 * P + t) * Wb + c] = gam1;
    __syncthreads();
    const int tn = (t + 1) & (P - 1);
    const R rho_n = sTop[(0 * P + tn) * Wb + c], alp_n = sTop[(1 * P + tn) * Wb + c],
            gam_n = sTop[(2 * P + tn) * Wb + c];
    Reduced<R> q = make_reduced<R>(ae, be, ce, re, qp, qq, qw, rho_n, alp_n, gam_n);
    __syncthreads();
    R *sL = small + c, *sD = small + P * Wb + c, *sU = small + 2 * P * Wb + c,
      *sRr = small + 3 * P * Wb + c;
    const R X = pcr_smem<R>(q, t, P, sL, sD, sU, sRr, Wb);
    R *sX = small + 4 * P * Wb;
    sX[t * Wb + c] = X;
    __syncthreads();
    const R Xm = sX[((t - 1) & (P - 1)) * Wb + c];

    if (K) {
        // Compensated state: as in line_sweep_kernel, the column's compensated
        // sum of delta (zero in exact arithmetic) is removed evenly and
        // hi + lo + delta - corr is formed in double-word arithmetic.
        R dprev = Xm;
        CSum<R> acc;
        for (int k = s; k < e; ++k) {
            const R d = sRho[ph(k)] - sAlp[ph(k)] * dprev - sGam[ph(k)] * X;
            sRho[ph(k)] = d;
            acc.add(d);
            dprev = d;
        }
        sRho[ph(e)] = X;
        acc.add(X);
        const double part = (double)acc.s + (double)acc.c;
        double *red = reinterpret_cast<double *>(small);  // PCR area, free now
        __syncthreads();
        red[t * Wb + c] = part;
        __syncthreads();
        double csum = 0.0;
        for (int k = 0; k < P; ++k) csum += red[k * Wb + c];  // same order in every thread of the column
        R ch, cl;
        split_f64(csum / (double)ny, ch, cl);
        if (active) {
            for (int k = s; k <= e; ++k) {
                const size_t o = (size_t)k * nx + ic;
                R hi, lo;
                dw_update(Tin[o], TinL[o], sRho[ph(k)], ch, cl, hi, lo);
                static_cast<R *>(J.Tout)[o] = hi;
                static_cast<R *>(J.ToutLo)[o] = lo;
                flag_nonfinite(args.err, hi);
            }
        }
    } else if (active) {
        R *out = static_cast<R *>(J.Tout);
        R dprev = Xm;
        for (int k0 = s; k0 <= e; k0 += UB) {
            R To[UB], Tw[UB] = {};
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                const int k = k0 + u <= e ? k0 + u : e;
                To[u] = Tin[(size_t)k * nx + ic];
                if (K) Tw[u] = TinL[(size_t)k * nx + ic];
            }
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                const int k = k0 + u;
                if (k > e) break;
                const R d = k < e ? sRho[ph(k)] - sAlp[ph(k)] * dprev - sGam[ph(k)] * X : X;
                dprev = d;
                if (K) {
                    R hi, lo;
                    kahan_add(To[u], Tw[u], d, hi, lo);
                    out[(size_t)k * nx + ic] = hi;
                    static_cast<R *>(J.ToutLo)[(size_t)k * nx + ic] = lo;
                    flag_nonfinite(args.err, hi);
                } else {
                    const R v = To[u] + d;
                    out[(size_t)k * nx + ic] = v;
                    flag_nonfinite(args.err, v);
                }
            }
        }
    }
}

// ======================================================= setup / utility

// Face coefficients of Section 2 (b averaged to faces by the plain mean) in FP64
// with explicit round-to-nearest operations (no contraction), then one
// rounding to the storage type.
template <typename C> __device__ __forceinline__ C to_store(double v);
template <> __device__ __forceinline__ double to_store<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __half to_store<__half>(double v) { return __double2half(v); }

template <typename B, typename C>
__global__ void face_coeffs_kernel(const B *__restrict__ bx, const B *__restrict__ by, int nx,
                                   int ny, int bc, double kappa, C *cxx, C *cxy, C *cyy, C *cyx,
                                   C *cyyT, C *cyxT)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= nx || j >= ny) return;
    const size_t o = (size_t)j * nx + i;
    const double omk = __dsub_rn(1.0, kappa);
    double vxx = 0.0, vxy = 0.0, vyy = 0.0, vyx = 0.0;
    const bool per = bc == 1;  // otherwise the boundary faces carry no flux
    if (per || i != nx - 1) {
        const size_t o1 = (size_t)j * nx + ((i + 1) % nx);
        const double fbx = __dmul_rn(0.5, __dadd_rn((double)bx[o], (double)bx[o1]));
        const double fby = __dmul_rn(0.5, __dadd_rn((double)by[o], (double)by[o1]));
        vxx = __dadd_rn(kappa, __dmul_rn(omk, __dmul_rn(fbx, fbx)));
        vxy = __dmul_rn(omk, __dmul_rn(fbx, fby));
    }
    if (per || j != ny - 1) {
        const size_t o1 = (size_t)((j + 1) % ny) * nx + i;
        const double fbx = __dmul_rn(0.5, __dadd_rn((double)bx[o], (double)bx[o1]));
        const double fby = __dmul_rn(0.5, __dadd_rn((double)by[o], (double)by[o1]));
        vyy = __dadd_rn(kappa, __dmul_rn(omk, __dmul_rn(fby, fby)));
        vyx = __dmul_rn(omk, __dmul_rn(fby, fbx));
    }
    cxx[o] = to_store<C>(vxx);
    cxy[o] = to_store<C>(vxy);
    cyy[o] = to_store<C>(vyy);
    cyx[o] = to_store<C>(vyx);
    if (cyyT) {
        const size_t oT = (size_t)i * ny + j;
        cyyT[oT] = to_store<C>(vyy);
        cyxT[oT] = to_store<C>(vyx);
    }
}

template <typename E>
__global__ void transpose_kernel(const E *__restrict__ in, E *__restrict__ out, int rows, int cols)
{
    __shared__ E tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

// Deterministic FP64 reductions: a fixed grid of TOTALS_BLOCKS blocks, each
// thread a fixed strided subset, fixed-order trees.
template <typename R>
__global__ void __launch_bounds__(256) totals_partial_kernel(const R *__restrict__ T, const R *__restrict__ Tlo,
                                                             size_t n, double *partials)
{
    __shared__ double ss[256], smin[256], smax[256], snf[256];
    double s = 0.0, lo = INFINITY, hi = -INFINITY, nf = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const double v = Tlo ? (double)T[k] + (double)Tlo[k] : (double)T[k];
        if (isfinite(v)) {
            s += v;
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        } else {
            nf += 1.0;
        }
    }
    ss[threadIdx.x] = s;
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    snf[threadIdx.x] = nf;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            ss[threadIdx.x] += ss[threadIdx.x + h];
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + h]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + h]);
            snf[threadIdx.x] += snf[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = ss[0];
        partials[gridDim.x + blockIdx.x] = smin[0];
        partials[2 * gridDim.x + blockIdx.x] = smax[0];
        partials[3 * gridDim.x + blockIdx.x] = snf[0];
    }
}

static __global__ void __launch_bounds__(32) totals_final_kernel(const double *partials, int nb,
                                                          double *result)
{
    if (threadIdx.x != 0) return;
    double s = 0.0, lo = INFINITY, hi = -INFINITY, nf = 0.0;
    for (int b = 0; b < nb; ++b) {
        s += partials[b];
        lo = fmin(lo, partials[nb + b]);
        hi = fmax(hi, partials[2 * nb + b]);
        nf += partials[3 * nb + b];
    }
    result[0] = s;
    result[1] = lo;
    result[2] = hi;
    result[3] = nf;
}

}  // namespace aniso
